"""GPU parity of SpMV (CSR/ELL/COO/hybrid x FP64/FP32/BF16), the format
conversions and the CSR plan against the CPU oracle, through the C ABI."""
import numpy as np
import pytest

import oracle as O
from gpu_util import bf16_round, check_spmv_f32, check_spmv_f64, dev, host, rows_subset
from paper_2006_14290_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FORMATS = ["csr", "ell", "coo", "hybrid", "sellp"]


def small_cases():
    rng = np.random.default_rng(2024)
    yield "laplace2d_64", I.laplace2d_5pt(64)
    yield "stencil27_12", I.stencil3d_27pt(12)
    yield "stencil7_17", I.stencil3d_7pt(17)
    yield "convdiff_9", I.convdiff3d_7pt(9, 10.0)
    yield "random_empty_unsorted", I.random_csr(3001, 2500, 0.004, rng, empty_rows=0.3, sort_cols=False)
    yield "dup_cols", I.rows_csr(rng.integers(0, 40, 777), 50, rng)
    yield "long_rows", I.rows_csr([3, 5000, 0, 2, 40000, 1, 1025, 1024, 7] + [2] * 3000, 60000, rng)
    yield "powerlaw_20k", I.powerlaw(20000, seed=1)
    yield "banded_5k", I.banded(5000, 16, 0.3, seed=2)
    yield "n1", I.rows_csr([3], 5, rng)
    # Segmented-reduction boundaries (8 entries per thread, 256 per warp, 1024
    # per COO tile): every thread ending a row on its last entry; rows ending
    # on warp and tile edges; empty rows right after a tile edge.
    yield "rows_of_8", I.rows_csr([8] * 4099, 3000, rng)
    # row ends at entries 256, 512, ..., 2048, 3072, 5120, ... (5 on tile edges, 16 on warp edges)
    yield "warp_tile_edges", I.rows_csr([256] * 4 + [1024, 1, 1023, 1025, 1023, 0, 255, 1, 0, 257, 255, 0, 512, 511, 1,
                                         2047, 1] + [8] * 32 + [7, 9] * 16 + [3, 253, 1024, 0, 0, 1], 4000, rng)
    yield "empty_after_tile_edge", I.rows_csr([1024, 0, 0, 1024, 0, 512, 512, 0, 3, 1021, 0] * 5, 2000, rng)


CASES = list(small_cases())


def make(G, A, fmt, dtype):
    vals = A.val if dtype == G.F64 else A.val.astype(np.float32)
    M = G.from_csr(A, G.F64 if dtype in (G.F64, G.BF16) else G.F32)
    if dtype == G.BF16:
        M = G.gko_matrix_convert_values(M, G.BF16)
    if fmt == "ell":
        M = G.gko_matrix_convert_to_ell(M, max_fill=1e9)
    elif fmt == "coo":
        M = G.gko_matrix_convert_to_coo(M)
    elif fmt == "hybrid":
        M = G.gko_matrix_convert_to_hybrid(M, -1)
    elif fmt == "sellp":
        M = G.gko_matrix_convert_to_sellp(M, 64, max_fill=1e9)
    return M


def values_for(G, A, dtype):
    if dtype == G.F64:
        return A.val
    if dtype == G.F32:
        return A.val.astype(np.float32).astype(np.float64)
    return bf16_round(A.val)


@pytest.mark.parametrize("name,A", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
def test_spmv_parity(gko, name, A, fmt, dt):
    G = gko
    dtype = {"f64": G.F64, "f32": G.F32, "bf16": G.BF16}[dt]
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, A.n_cols)
    y0 = rng.uniform(-1, 1, A.n_rows)
    M = make(G, A, fmt, dtype)
    for alpha, beta in [(1.0, 0.0), (-0.75, 1.5)]:
        if dtype == G.F64:
            yd = dev(y0)
            G.gko_spmv(alpha, M, dev(x), beta, yd)
            check_spmv_f64(host(yd), A, x, alpha, beta, y0)
        else:
            x32 = x.astype(np.float32)
            yd = dev(y0, np.float32)
            G.gko_spmv(alpha, M, dev(x32), beta, yd)
            check_spmv_f32(host(yd), A, x32.astype(np.float64), alpha, beta, y0.astype(np.float32).astype(np.float64),
                           values_for(G, A, dtype))


@pytest.mark.parametrize("name,A", CASES, ids=[c[0] for c in CASES])
def test_conversions_bit_exact(gko, name, A):
    G = gko
    M = G.from_csr(A)
    ex = M.export()
    np.testing.assert_array_equal(ex["row_ptr"], A.row_ptr)
    np.testing.assert_array_equal(ex["col"], A.col)
    assert ex["val"].tobytes() == A.val.tobytes()

    E = G.gko_matrix_convert_to_ell(M, max_fill=1e9).export()
    Eo = O.csr_to_ell(A)
    assert (E["ell_width"], E["ell_stride"]) == (Eo.K, Eo.stride)
    np.testing.assert_array_equal(E["ell_col"], Eo.col)
    assert E["ell_val"].tobytes() == Eo.val.tobytes()

    C = G.gko_matrix_convert_to_coo(M).export()
    Co = O.csr_to_coo(A)
    np.testing.assert_array_equal(C["coo_row"], Co.row)
    np.testing.assert_array_equal(C["coo_col"], Co.col)
    assert C["coo_val"].tobytes() == Co.val.tobytes()

    for K in (-1, 0, 2, 5):
        H = G.gko_matrix_convert_to_hybrid(M, K).export()
        Ho = O.csr_to_hybrid(A, K)
        assert H["ell_width"] == Ho.ell.K
        np.testing.assert_array_equal(H["ell_col"], Ho.ell.col)
        assert H["ell_val"].tobytes() == Ho.ell.val.tobytes()
        np.testing.assert_array_equal(H["coo_row"], Ho.coo.row)
        np.testing.assert_array_equal(H["coo_col"], Ho.coo.col)
        assert H["coo_val"].tobytes() == Ho.coo.val.tobytes()

    for C in (32, 64, 128, 256):
        S = G.gko_matrix_convert_to_sellp(M, C, max_fill=1e9).export()
        So = O.csr_to_sellp(A, C=C)
        assert S["ell_stride"] == C and S["coo_nnz"] == So.sets[-1] * C
        np.testing.assert_array_equal(S["sets"], So.sets)
        np.testing.assert_array_equal(S["ell_col"], So.col)
        assert S["ell_val"].tobytes() == So.val.tobytes()


def test_value_conversions_round_to_nearest(gko):
    G = gko
    A = I.powerlaw(3000, seed=5)
    M = G.from_csr(A)
    v32 = G.gko_matrix_convert_values(M, G.F32).export()["val"]
    assert v32.tobytes() == A.val.astype(np.float32).tobytes()
    vb = G.gko_matrix_convert_values(M, G.BF16).export()["val"]
    ref = bf16_round(A.val).astype(np.float32).view(np.uint32) >> 16
    np.testing.assert_array_equal(vb.astype(np.uint32), ref)


def test_plan_histogram_and_split(gko):
    G = gko
    for A in (I.powerlaw(20000, seed=1), I.laplace2d_5pt(64), I.rows_csr([0, 1, 2, 3, 4, 2000, 70000], 10, np.random.default_rng(0))):
        p = G.from_csr(A).plan()
        L = A.row_lengths()
        cls = np.where(L == 0, 0, np.floor(np.log2(np.maximum(L, 1))).astype(int) + 1)
        np.testing.assert_array_equal(p["hist"], np.bincount(cls, minlength=33))
        if L.max() <= 4 * L.mean() + 1:  # regular: row-block kernel, nothing split
            m = L.mean()
            S = 1
            while S < 8 and (128 // S) * m > 0.9 * 1024:
                S *= 2
            R = 1
            while R < 4 and (128 // S) * 2 * R * m <= 1024:
                R *= 2
            assert (p["kernel"], p["subwarp"], p["rows_per_subwarp"], p["stage_cap"], p["n_long_rows"]) == \
                (1, S, R, 1024, 0)
            continue
        assert p["kernel"] == 3 and p["n_long_rows"] == 0  # skewed: nonzero split
        M = G.from_csr(A)
        M.set_plan(0, 8, 2)
        p = M.plan()
        longs = L[L > 32 * 8]
        assert p["kernel"] == 0 and p["long_threshold"] == 256
        assert p["n_long_rows"] == longs.size
        assert p["n_long_chunks"] == int(np.sum((longs + 1023) // 1024))


PLANS = ([(0, S, R, 2048) for S in (1, 2, 4, 8, 16, 32) for R in (1, 2, 4)]
         + [(1, S, R, cap) for S in (1, 2, 4, 8) for R in (1, 2, 4) for cap in (512, 2048)]
         + [(1, 1, 4, 8192), (1, 2, 1, 1024), (2, 1, 1, 2048), (3, 1, 1, 1024)])


@pytest.mark.parametrize("kernel,S,R,cap", PLANS)
@pytest.mark.parametrize("mat", ["powerlaw", "banded"])
def test_every_plan_matches_oracle(gko, kernel, S, R, cap, mat):
    """Every subwarp plan and every row-block plan (lanes per row, interleaved
    rows, stage capacity), including row blocks that need many stages."""
    G = gko
    A = I.powerlaw(30000, seed=3) if mat == "powerlaw" else I.banded(40000, 200, 0.7, seed=5)
    M = G.from_csr(A)
    M.set_plan(kernel, S, R, cap)
    p = M.plan()
    assert (p["kernel"], p["subwarp"], p["rows_per_subwarp"]) == (kernel, S, R)
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, A.n_cols)
    y0 = rng.uniform(-1, 1, A.n_rows)
    yd = dev(y0)
    G.gko_spmv(2.0, M, dev(x), -1.0, yd)
    check_spmv_f64(host(yd), A, x, 2.0, -1.0, y0)


def empty_run_cases():
    rng = np.random.default_rng(31)
    # tiles spanning thousands of empty rows (row pointers read from global
    # memory), empty rows before the first and after the last nonzero
    yield "empty_runs", I.rows_csr([0] * 700 + [3] + [0] * 5000 + [2] * 10 + [0] * 3000 + [1500, 1] + [0] * 2600
                                   + [7] * 300 + [0] * 9000, 3000, rng)
    yield "one_row", I.rows_csr([5000], 7000, rng)
    yield "all_single", I.rows_csr([1] * 5000, 5000, rng)


SEG_CASES = CASES + list(empty_run_cases())


@pytest.mark.parametrize("name,A", SEG_CASES, ids=[c[0] for c in SEG_CASES])
@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
def test_nonzero_split_plan(gko, name, A, dt):
    """CSR kernel 3 (nonzero split) on every case matrix, both alpha/beta
    settings, all value types."""
    G = gko
    dtype = {"f64": G.F64, "f32": G.F32, "bf16": G.BF16}[dt]
    M = make(G, A, "csr", dtype)
    M.set_plan(3, 1, 1, 1024)
    assert M.plan()["kernel"] == 3
    rng = np.random.default_rng(8)
    x = rng.uniform(-1, 1, A.n_cols)
    y0 = rng.uniform(-1, 1, A.n_rows)
    for alpha, beta in [(1.0, 0.0), (-0.75, 1.5)]:
        if dtype == G.F64:
            yd = dev(y0)
            G.gko_spmv(alpha, M, dev(x), beta, yd)
            check_spmv_f64(host(yd), A, x, alpha, beta, y0)
        else:
            x32 = x.astype(np.float32)
            yd = dev(y0, np.float32)
            G.gko_spmv(alpha, M, dev(x32), beta, yd)
            check_spmv_f32(host(yd), A, x32.astype(np.float64), alpha, beta, y0.astype(np.float32).astype(np.float64),
                           values_for(G, A, dtype))


@pytest.mark.parametrize("C", [32, 128, 256])
@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
def test_sellp_slice_sizes(gko, C, dt):
    """SELL-P at every slice height; ragged last slice, empty rows."""
    G = gko
    rng = np.random.default_rng(21)
    L = rng.integers(0, 30, 5003)
    L[700:1100] = 0
    A = I.rows_csr(L, 4000, rng)
    dtype = {"f64": G.F64, "f32": G.F32, "bf16": G.BF16}[dt]
    M = G.from_csr(A, G.F64 if dtype in (G.F64, G.BF16) else G.F32)
    if dtype == G.BF16:
        M = G.gko_matrix_convert_values(M, G.BF16)
    S = G.gko_matrix_convert_to_sellp(M, C)
    x = rng.uniform(-1, 1, A.n_cols)
    y0 = rng.uniform(-1, 1, A.n_rows)
    if dtype == G.F64:
        yd = dev(y0)
        G.gko_spmv(0.5, S, dev(x), 2.0, yd)
        check_spmv_f64(host(yd), A, x, 0.5, 2.0, y0)
    else:
        x32 = x.astype(np.float32)
        yd = dev(y0, np.float32)
        G.gko_spmv(0.5, S, dev(x32), 2.0, yd)
        check_spmv_f32(host(yd), A, x32.astype(np.float64), 0.5, 2.0, y0.astype(np.float32).astype(np.float64),
                       values_for(G, A, dtype))


def test_sellp_rejects_bad_slice_and_padding(gko):
    G = gko
    M = G.from_csr(I.powerlaw(20000, seed=1))
    with pytest.raises(G.GkoError) as e:
        G.gko_matrix_convert_to_sellp(M)  # slices of 64 random power-law rows: padding over 8x nnz
    assert e.value.status == G.FORMAT_UNSUITABLE
    for bad in (16, 48, 512):
        with pytest.raises(G.GkoError) as e:
            G.gko_matrix_convert_to_sellp(M, bad, max_fill=1e9)
        assert e.value.status == G.INVALID_ARG


def test_coo_plan_defaults(gko):
    """COO starts on the segmented reduction with the CSR histogram; the
    row-block schedule is opt-in."""
    G = gko
    for A in (I.laplace2d_5pt(64), I.stencil3d_27pt(10), I.banded(5000, 16, 0.3, seed=2), I.powerlaw(20000, seed=1)):
        M = G.from_csr(A)
        pc, po = M.plan(), G.gko_matrix_convert_to_coo(M).plan()
        assert po["kernel"] == 0
        np.testing.assert_array_equal(po["hist"], pc["hist"])


COO_PLANS = ([(1, S, R, cap) for S in (1, 2, 4, 8) for R in (1, 2, 4) for cap in (512, 4096)]
             + [(1, 1, 1, 1024), (0, 1, 1, 2048)])


def _coo_plan_matrix(mat):
    rng = np.random.default_rng(12)
    if mat == "powerlaw":  # rows far longer than a stage: row blocks over many stages
        return I.powerlaw(30000, seed=3)
    if mat == "banded":
        return I.banded(40000, 200, 0.7, seed=5)
    # empty rows (also whole empty row blocks), unsorted columns, ragged last block
    L = rng.integers(0, 9, 20011)
    L[100:700] = 0
    L[-3:] = 0
    return I.rows_csr(L, 9000, rng)


@pytest.mark.parametrize("kernel,S,R,cap", COO_PLANS)
@pytest.mark.parametrize("mat", ["powerlaw", "banded", "gaps"])
def test_every_coo_plan_matches_oracle(gko, kernel, S, R, cap, mat):
    """Row-block COO under every lanes/rows/stage choice, on skewed rows
    spanning many stages, on dense bands, and on matrices with empty rows and
    empty row blocks; kernel 0 is the segmented reduction."""
    G = gko
    A = _coo_plan_matrix(mat)
    M = G.gko_matrix_convert_to_coo(G.from_csr(A))
    M.set_plan(kernel, S, R, cap)
    p = M.plan()
    assert p["kernel"] == kernel
    if kernel == 1:
        assert (p["subwarp"], p["rows_per_subwarp"], p["stage_cap"]) == (S, R, cap)
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, A.n_cols)
    y0 = rng.uniform(-1, 1, A.n_rows)
    for alpha, beta in [(1.0, 0.0), (2.0, -1.0)]:
        yd = dev(y0)
        G.gko_spmv(alpha, M, dev(x), beta, yd)
        check_spmv_f64(host(yd), A, x, alpha, beta, y0)


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_coo_rowblock_low_precision_shares_plan(gko, dt):
    """Value conversions of a row-block COO handle keep its row-block starts."""
    G = gko
    A = I.stencil3d_27pt(14)
    M = G.gko_matrix_convert_to_coo(G.from_csr(A))
    M.set_plan(1, 2, 2, 512)
    L = G.gko_matrix_convert_values(M, G.F32 if dt == "f32" else G.BF16)
    assert L.plan()["kernel"] == 1
    x32 = np.random.default_rng(3).uniform(-1, 1, A.n_cols).astype(np.float32)
    yd = dev(np.zeros(A.n_rows), np.float32)
    G.gko_spmv(1.0, L, dev(x32), 0.0, yd)
    vals = A.val.astype(np.float32).astype(np.float64) if dt == "f32" else bf16_round(A.val)
    check_spmv_f32(host(yd), A, x32.astype(np.float64), 1.0, 0.0, None, vals)


def test_coo_plan_rejects_bad_values(gko):
    G = gko
    M = G.gko_matrix_convert_to_coo(G.from_csr(I.laplace2d_5pt(8)))
    for bad in [(1, 16, 1, 1024), (1, 1, 3, 1024), (1, 1, 1, 8192), (1, 1, 1, 768), (3, 1, 1, 1024)]:
        with pytest.raises(G.GkoError) as e:
            M.set_plan(*bad)
        assert e.value.status == G.INVALID_ARG


def test_edge_cases(gko):
    G = gko
    # zero rows
    Z = I.Csr(0, 5, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    M = G.from_csr(Z)
    G.gko_spmv(1.0, M, dev(np.ones(5)), 0.0, dev(np.zeros(1)))
    # no nonzeros: y = beta*y (beta = 0 writes zeros without reading NaN)
    E = I.Csr(10, 10, np.zeros(11, np.int32), np.zeros(0, np.int32), np.zeros(0))
    for fmt in FORMATS:
        M = make(G, E, fmt, G.F64)
        yd = dev(np.arange(10.0))
        G.gko_spmv(1.0, M, dev(np.ones(10)), 3.0, yd)
        np.testing.assert_array_equal(host(yd), 3.0 * np.arange(10.0))
        yd = dev(np.full(10, np.nan))
        G.gko_spmv(1.0, M, dev(np.ones(10)), 0.0, yd)
        np.testing.assert_array_equal(host(yd), np.zeros(10))


@pytest.mark.parametrize("fmt", FORMATS)
def test_nan_semantics(gko, fmt):
    G = gko
    A = I.laplace2d_5pt(16)
    M = make(G, A, fmt, G.F64)
    x = np.ones(256)
    x[37] = np.nan
    y0 = np.full(256, np.nan)
    yd = dev(y0)
    G.gko_spmv(1.0, M, dev(x), 0.0, yd)
    check_spmv_f64(host(yd), A, x, 1.0, 0.0, None)
    yd = dev(np.ones(256))
    G.gko_spmv(0.0, M, dev(x), 1.0, yd)
    check_spmv_f64(host(yd), A, x, 0.0, 1.0, np.ones(256))


def test_invalid_inputs_rejected(gko):
    G = gko
    A = I.laplace2d_5pt(4)
    bad_col = A.col.copy()
    bad_col[3] = 16
    with pytest.raises(G.GkoError) as e:
        G.gko_matrix_create_csr(16, 16, A.row_ptr, bad_col, A.val)
    assert e.value.status == G.INVALID_ARG
    bad_rp = A.row_ptr.copy()
    bad_rp[5], bad_rp[6] = bad_rp[6], bad_rp[5]
    with pytest.raises(G.GkoError):
        G.gko_matrix_create_csr(16, 16, bad_rp, A.col, A.val)
    with pytest.raises(G.GkoError) as e:
        G.gko_matrix_convert_to_ell(G.from_csr(I.powerlaw(20000, seed=1)))
    assert e.value.status == G.FORMAT_UNSUITABLE
    M = G.from_csr(A)
    import torch
    with pytest.raises(G.GkoError):
        G.gko_spmv(1.0, M, torch.ones(16, device="cuda", dtype=torch.float32), 0.0,
                   torch.zeros(16, device="cuda", dtype=torch.float32))


@pytest.mark.parametrize("fmt", FORMATS)
def test_deterministic(gko, fmt):
    G = gko
    A = I.powerlaw(50000, seed=9)
    M = make(G, A, fmt, G.F64) if fmt != "ell" else make(G, I.banded(20000, 40, 0.5, seed=1), fmt, G.F64)
    n = M.info()["n_cols"]
    x = dev(np.random.default_rng(0).uniform(-1, 1, n))
    outs = []
    for _ in range(3):
        yd = dev(np.zeros(M.info()["n_rows"]))
        G.gko_spmv(1.0, M, x, 0.0, yd)
        outs.append(host(yd).tobytes())
    assert outs[0] == outs[1] == outs[2]


def _full_size(name):
    if name == "stencil27_128":
        return I.stencil3d_27pt(128)
    if name == "powerlaw_1m":
        return I.powerlaw(1_000_000, seed=0)
    return I.banded(1_000_000, 64, 0.3, seed=0)


@pytest.mark.slow
@pytest.mark.parametrize("name", ["stencil27_128", "powerlaw_1m", "banded_1m"])
def test_full_size_sampled(gko, name):
    """Bench-size matrices in the bench's launch configuration, checked on
    sampled rows (plus every long row) against the oracle."""
    G = gko
    A = _full_size(name)
    rng = np.random.default_rng(11)
    x = rng.uniform(-1, 1, A.n_cols)
    L = A.row_lengths()
    idx = np.unique(np.concatenate([rng.integers(0, A.n_rows, 4000), [0, A.n_rows - 1],
                                    np.flatnonzero(L > 256)[:2000]]))
    sub = rows_subset(A, idx)
    M64 = G.from_csr(A)
    formats = [("csr", M64), ("coo", G.gko_matrix_convert_to_coo(M64)), ("hybrid", G.gko_matrix_convert_to_hybrid(M64))]
    if name != "powerlaw_1m":
        formats.append(("ell", G.gko_matrix_convert_to_ell(M64)))
        formats.append(("sellp", G.gko_matrix_convert_to_sellp(M64)))
    xd = dev(x)
    for fmt, M in formats:
        yd = dev(np.zeros(A.n_rows))
        G.gko_spmv(1.0, M, xd, 0.0, yd)
        check_spmv_f64(host(yd)[idx], sub, x, 1.0, 0.0, None)
        del M
    M32 = G.from_csr(A, G.F32)
    x32 = x.astype(np.float32)
    yd = dev(np.zeros(A.n_rows, np.float32))
    G.gko_spmv(1.0, M32, dev(x32), 0.0, yd)
    check_spmv_f32(host(yd)[idx], sub, x32.astype(np.float64), 1.0, 0.0, None, sub.val.astype(np.float32).astype(np.float64))


def test_memory_budget_refuses_and_recovers(gko):
    G = gko
    A = I.laplace2d_5pt(64)
    used = G.memory_in_use()
    G.set_memory_budget(used + 1024)
    try:
        with pytest.raises(G.GkoError) as e:
            G.from_csr(A)
        assert e.value.status == G.BUDGET_EXCEEDED
        assert G.memory_in_use() == used
    finally:
        G.set_memory_budget(0)
    M = G.from_csr(A)
    assert G.memory_in_use() > used
    del M


@pytest.mark.parametrize("fmt", ["csr", "coo"])
def test_spmv_host_buffers(gko, fmt):
    """gko_spmv_host: host x and y (pinned), copies in stream order; equals
    the oracle for beta = 0 and beta != 0."""
    import torch

    G = gko
    A = I.banded(3000, 12, 0.4, seed=4)
    M = make(G, A, fmt, G.F64)
    rng = np.random.default_rng(8)
    x = rng.uniform(-1, 1, A.n_cols)
    y0 = rng.uniform(-1, 1, A.n_rows)
    xh = torch.from_numpy(x).pin_memory()
    xd = torch.empty(A.n_cols, dtype=torch.float64, device="cuda")
    yd = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
    for alpha, beta in [(1.0, 0.0), (-2.0, 0.5)]:
        yh = torch.from_numpy(y0.copy()).pin_memory()
        G.gko_spmv_host(alpha, M, xh, beta, yh, xd, yd)
        torch.cuda.synchronize()
        check_spmv_f64(yh.numpy(), A, x, alpha, beta, y0)


@pytest.mark.parametrize("fmt", ["csr", "coo"])
@pytest.mark.parametrize("mat", ["banded", "powerlaw"])
def test_tune_sets_a_valid_plan(gko, fmt, mat):
    """The plan autotuner leaves the handle on the plan it reports, and SpMV
    on that plan matches the oracle (FP64 and an FP32 copy)."""
    import torch

    G = gko
    A = I.banded(30000, 24, 0.5, seed=6) if mat == "banded" else I.powerlaw(30000, seed=7)
    M = make(G, A, fmt, G.F64)
    x = np.random.default_rng(2).uniform(-1, 1, A.n_cols)
    xd, yd = dev(x), torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
    k0 = M.plan()["kernel"]
    k, S, R, cap, ms = M.tune(xd, yd, reps=1, keep_kernel=True)
    assert k == k0 and M.plan()["kernel"] == k0
    k, S, R, cap, ms = M.tune(xd, yd, reps=1)
    p = M.plan()
    assert p["kernel"] == k and ms > 0
    if k == 1:
        assert (p["subwarp"], p["rows_per_subwarp"], p["stage_cap"]) == (S, R, cap)
    yd = dev(np.zeros(A.n_rows))
    G.gko_spmv(1.0, M, xd, 0.0, yd)
    check_spmv_f64(host(yd), A, x, 1.0, 0.0, None)
    M32 = G.gko_matrix_convert_values(M, G.F32)
    x32 = x.astype(np.float32)
    M32.tune(dev(x32), torch.empty(A.n_rows, dtype=torch.float32, device="cuda"), reps=1)
    yd = dev(np.zeros(A.n_rows), np.float32)
    G.gko_spmv(1.0, M32, dev(x32), 0.0, yd)
    check_spmv_f32(host(yd), A, x32.astype(np.float64), 1.0, 0.0, None, A.val.astype(np.float32).astype(np.float64))


def test_tune_refuses_other_formats(gko):
    G = gko
    A = I.laplace2d_5pt(8)
    E = G.gko_matrix_convert_to_ell(G.from_csr(A))
    import torch
    with pytest.raises(G.GkoError) as e:
        E.tune(dev(np.ones(64)), torch.empty(64, dtype=torch.float64, device="cuda"))
    assert e.value.status == G.NOT_SUPPORTED
