"""GPU parity of the batched persistent CG against per-system oracle CG."""
import numpy as np
import pytest

import oracle as O
from gpu_util import dev, host
from paper_2006_14290_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def batch_problem(count, seed=0, extra_sides=(8, 64, 11)):
    sides = list(I.batch_sides(count, seed=seed)) + list(extra_sides)
    systems, bs = [], []
    for i, sd in enumerate(sides):
        A, b = I.batch_system(i, int(sd), seed=seed)
        systems.append(A)
        bs.append(b)
    return systems, bs


def concat(v):
    return np.concatenate([np.asarray(a, np.float64) for a in v])


@pytest.mark.parametrize("storage", ["csr", "ell"])
@pytest.mark.parametrize("threads", [256, 512, 1024])
@pytest.mark.parametrize("threshold", [0, 64, 144, 256])
def test_batch_cg_matches_oracle(gko, threshold, threads, storage):
    """Every schedule (warp threshold x threads per block x CSR or ELL
    storage) against the per-system oracle CG."""
    G = gko
    systems, bs = batch_problem(120)
    bs[5] = np.zeros_like(bs[5])  # a zero right-hand side
    B = G.Batch(systems)
    B.set_schedule(threshold, threads, G.BATCH_ELL if storage == "ell" else G.BATCH_CSR)
    b = concat(bs)
    xd = dev(np.zeros(b.size))
    code, it, rr, st = B.cg(dev(b), xd, 1e-12, 20000)
    assert code == G.OK and np.all(st == G.OK)
    x = host(xd)
    off = B.row_off
    for i in list(range(0, len(systems), 9)) + [5, len(systems) - 3, len(systems) - 2, len(systems) - 1]:
        A = systems[i]
        xi = x[off[i]:off[i + 1]]
        if i == 5:
            assert it[i] == 0 and np.all(xi == 0) and rr[i] == 0
            continue
        xo, ro = O.cg(A, bs[i], tol=1e-12, maxit=20000)
        assert ro.status == 0
        assert np.linalg.norm(xi - xo) <= 1e-8 * np.linalg.norm(xo), i
        assert abs(int(it[i]) - ro.iterations) <= max(2, 0.1 * ro.iterations), (i, it[i], ro.iterations)
        true = np.linalg.norm(bs[i] - O.spmv_csr(A, xi)) / np.linalg.norm(bs[i])
        assert true <= 1.01e-12 and abs(true - rr[i]) <= 1e-14


def test_batch_deterministic_graph_replay_and_x0(gko):
    G = gko
    systems, bs = batch_problem(60, seed=3)
    B = G.Batch(systems)
    b = dev(concat(bs))
    x0 = np.random.default_rng(2).uniform(-1, 1, B.total_rows)
    outs = []
    for _ in range(3):  # first call captures the graph, later calls replay it
        xd = dev(x0)
        code, it, rr, st = B.cg(b, xd, 1e-11, 20000)
        assert code == G.OK
        outs.append((host(xd).tobytes(), it.tobytes()))
    assert outs[0] == outs[1] == outs[2]


def test_batch_fp32_storage_and_caps(gko):
    G = gko
    systems, bs = batch_problem(40, seed=4)
    B = G.Batch(systems, storage=G.F32)
    b = concat(bs)
    xd = dev(np.zeros(b.size))
    code, it, rr, st = B.cg(dev(b), xd, 1e-10, 20000)
    assert code == G.OK
    x = host(xd)
    for i in range(0, len(systems), 7):
        A = systems[i]
        A32 = I.Csr(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64))
        xi = x[B.row_off[i]:B.row_off[i + 1]]
        true32 = np.linalg.norm(bs[i] - O.spmv_csr(A32, xi)) / np.linalg.norm(bs[i])
        assert true32 <= 1.01e-10
    xd = dev(np.zeros(b.size))
    code, it, rr, st = B.cg(dev(b), xd, 1e-14, 3)
    assert code == G.NOT_CONVERGED and np.all(it == 3) and np.all(st == G.NOT_CONVERGED)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_batch_stores_the_systems_it_was_given(gko, storage):
    """gko_batch_create_systems packs per-system CSR arrays itself: the
    exported offsets, row pointers and columns equal the concatenation, and
    the values equal the FP64 input (F64) or its round-to-nearest FP32
    rounding (F32 storage, rounded on the device) byte for byte."""
    G = gko
    systems, _ = batch_problem(50, seed=6)
    B = G.Batch(systems, storage=G.F64 if storage == "f64" else G.F32)
    ro, no, rp, col, val = B.export()
    rows = [S.n_rows for S in systems]
    nnzs = [int(S.row_ptr[-1]) for S in systems]
    assert ro.tolist() == [sum(rows[:i]) for i in range(len(rows) + 1)]
    assert no.tolist() == [sum(nnzs[:i]) for i in range(len(nnzs) + 1)]
    assert rp.tobytes() == np.concatenate([np.asarray(S.row_ptr, np.int32) for S in systems]).tobytes()
    assert col.tobytes() == np.concatenate([np.asarray(S.col, np.int32) for S in systems]).tobytes()
    v64 = np.concatenate([np.asarray(S.val, np.float64) for S in systems])
    want = v64 if storage == "f64" else v64.astype(np.float32)
    assert val.dtype == want.dtype and val.tobytes() == want.tobytes()


def test_batch_tuner_and_invalid_input(gko):
    G = gko
    systems, bs = batch_problem(200, seed=5)
    B = G.Batch(systems)
    b = dev(concat(bs))
    x0 = dev(np.zeros(B.total_rows))
    t = B.tune(b, x0, 1e-10, 20000)
    assert t["warp_rows"] in (0, 64, 144, 256) and t["threads"] in (256, 512, 1024) and t["ms"] > 0
    inf = B.info()
    assert (inf["warp_rows"], inf["threads"], inf["storage"]) == (t["warp_rows"], t["threads"], t["storage"])
    assert np.all(host(x0) == 0)
    bad = I.laplace2d_5pt(4)
    bad.col = bad.col.copy()
    bad.col[0] = 99
    with pytest.raises(G.GkoError):
        G.Batch([bad])


@pytest.mark.slow
def test_batch_full_size_4096(gko):
    """The batched workload of the benchmark: 4096 systems, sides in [8, 64]."""
    G = gko
    sides = I.batch_sides(4096)
    systems, bs = [], []
    for i, sd in enumerate(sides):
        A, b = I.batch_system(i, int(sd))
        systems.append(A)
        bs.append(b)
    B = G.Batch(systems)
    assert B.info()["total_rows"] == 3914078 and B.info()["total_nnz"] == 19132534
    b = concat(bs)
    xd = dev(np.zeros(b.size))
    code, it, rr, st = B.cg(dev(b), xd, 1e-10, 20000)
    assert code == G.OK and np.all(rr <= 1e-10)
    x = host(xd)
    for i in np.random.default_rng(0).choice(4096, 12, replace=False):
        A = systems[i]
        xi = x[B.row_off[i]:B.row_off[i + 1]]
        true = np.linalg.norm(bs[i] - O.spmv_csr(A, xi)) / np.linalg.norm(bs[i])
        assert true <= 1.01e-10
        xo, ro = O.cg(A, bs[i], tol=1e-10, maxit=20000)
        assert abs(int(it[i]) - ro.iterations) <= max(2, 0.1 * ro.iterations)


def test_batch_storages_give_identical_results(gko):
    """ELL storage keeps every row's entries in storage order, so the batch
    solved from it is bit-identical to the CSR run, at every group size."""
    G = gko
    # 5-point systems: boundary rows are shorter, so ELL pads them
    systems, bs = batch_problem(80, seed=7, extra_sides=(64, 8, 9, 33))
    B = G.Batch(systems)
    b = dev(concat(bs))
    outs = {}
    for threads in (256, 1024):
        for st in (G.BATCH_CSR, G.BATCH_ELL):
            B.set_schedule(64, threads, st)
            xd = dev(np.zeros(B.total_rows))
            code, it, rr, stt = B.cg(b, xd, 1e-11, 20000)
            assert code == G.OK
            outs[(threads, st)] = (host(xd).tobytes(), it.tobytes())
    for threads in (256, 1024):
        assert outs[(threads, G.BATCH_CSR)] == outs[(threads, G.BATCH_ELL)]


@pytest.mark.parametrize("storage", ["csr", "ell"])
@pytest.mark.parametrize("threads", [256, 512, 1024])
@pytest.mark.parametrize("threshold", [0, 144, 256])
def test_batch_mixed_reliable_matches_oracle(gko, threshold, threads, storage):
    """Mixed precision (FP32 recurrences, reliable updates) on every schedule
    against the oracle's reliable-update CG per system: both sides to 1e-12,
    solutions within 1e-8 of each other and of the FP64 oracle CG, the
    reported residual the true one, iteration counts within 15% (the GPU
    applies FP64 scalars to FP32 vectors as float pairs)."""
    G = gko
    systems, bs = batch_problem(120)
    bs[5] = np.zeros_like(bs[5])
    B = G.Batch(systems)
    B.set_schedule(threshold, threads, G.BATCH_ELL if storage == "ell" else G.BATCH_CSR)
    B.set_precision(G.PRECISION_MIXED_F32)
    b = concat(bs)
    xd = dev(np.zeros(b.size))
    code, it, rr, st = B.cg(dev(b), xd, 1e-12, 20000)
    up = B.last_updates()
    assert code == G.OK and np.all(st == G.OK)
    x = host(xd)
    off = B.row_off
    picks = list(range(0, len(systems), 9)) + [5, len(systems) - 3, len(systems) - 2, len(systems) - 1]
    xr, itr, upr, rrr, str_ = O.batch_cg_reliable([systems[i] for i in picks], [bs[i] for i in picks], tol=1e-12,
                                                  maxit=20000)
    for j, i in enumerate(picks):
        A = systems[i]
        xi = x[off[i]:off[i + 1]]
        if i == 5:
            assert it[i] == 0 and up[i] == 0 and np.all(xi == 0) and rr[i] == 0
            continue
        assert str_[j] == 0 and up[i] >= 1
        assert np.linalg.norm(xi - xr[j]) <= 1e-8 * np.linalg.norm(xr[j]), i
        xo, _ = O.cg(A, bs[i], tol=1e-12, maxit=20000)
        assert np.linalg.norm(xi - xo) <= 1e-8 * np.linalg.norm(xo), i
        assert abs(int(it[i]) - int(itr[j])) <= max(3, 0.15 * itr[j]), (i, it[i], itr[j])
        true = np.linalg.norm(bs[i] - O.spmv_csr(A, xi)) / np.linalg.norm(bs[i])
        assert true <= 1.01e-12 and abs(true - rr[i]) <= 1e-14


def test_batch_mixed_reliable_options_storage_and_caps(gko):
    """FP32 storage (the recurrences and the replaced residuals both use the
    stored FP32 values), deterministic replay, x0, switching back to FP64
    (update counts read zero), the iteration cap and bad arguments."""
    G = gko
    systems, bs = batch_problem(40, seed=4)
    b = concat(bs)
    B = G.Batch(systems, storage=G.F32)
    B.set_precision(G.PRECISION_MIXED_F32, 0.05)
    outs = []
    for _ in range(2):
        xd = dev(np.zeros(b.size))
        code, it, rr, st = B.cg(dev(b), xd, 1e-10, 20000)
        assert code == G.OK
        outs.append(host(xd).tobytes())
    assert outs[0] == outs[1]
    x = host(xd)
    off = B.row_off
    for i in range(0, len(systems), 7):
        A = systems[i]
        A32 = I.Csr(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64))
        xi = x[off[i]:off[i + 1]]
        assert np.linalg.norm(bs[i] - O.spmv_csr(A32, xi)) <= 1.01e-10 * np.linalg.norm(bs[i])
    x0 = np.random.default_rng(9).uniform(-1, 1, B.total_rows)
    xd = dev(x0)
    code, it, rr, st = B.cg(dev(b), xd, 1e-10, 20000)
    assert code == G.OK
    xd = dev(np.zeros(b.size))
    code, it, rr, st = B.cg(dev(b), xd, 1e-14, 3)
    assert code == G.NOT_CONVERGED and np.all(it <= 3)
    x = host(xd)
    for i in range(0, len(systems), 7):
        A32 = I.Csr(systems[i].n_rows, systems[i].n_cols, systems[i].row_ptr, systems[i].col,
                    systems[i].val.astype(np.float32).astype(np.float64))
        xi = x[off[i]:off[i + 1]]
        true = np.linalg.norm(bs[i] - O.spmv_csr(A32, xi)) / np.linalg.norm(bs[i])
        assert abs(true - rr[i]) <= 1e-12
    B.set_precision(G.PRECISION_F64)
    code, it, rr, st = B.cg(dev(b), dev(np.zeros(b.size)), 1e-10, 20000)
    assert code == G.OK and np.all(B.last_updates() == 0)
    for bad in ((G.PRECISION_MIXED_BF16, 0.1), (G.PRECISION_MIXED_F32, 1.0), (G.PRECISION_MIXED_F32, -0.5)):
        with pytest.raises(G.GkoError):
            B.set_precision(*bad)
