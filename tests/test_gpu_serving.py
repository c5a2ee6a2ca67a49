"""The serving loop: continuous batching over resident matrices.

Checks that every result is the same alone and in the mix (bitwise, since
all kernels are deterministic), that requests overlap on the device, that
the memory budget gates admission and rejects oversize requests, and that
malformed requests are refused on the host."""
import numpy as np
import pytest

import oracle as O
from paper_2006_14290_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def pool(G):
    rng = np.random.default_rng(0)
    mats = []
    for side in (10, 16, 24, 40):
        mats.append(("cg", I.varcoef3d_7pt(side, rng)))
    for side, P in ((10, 3.0), (16, 8.0), (20, 1.0)):
        mats.append(("bicgstab", I.convdiff3d_7pt(side, P)))
    return mats


def test_results_same_alone_and_in_the_mix(gko):
    G = gko
    mats = pool(G)
    handles = [G.from_csr(A) for _, A in mats]
    rng = np.random.default_rng(1)
    reqs = []
    for k in range(28):
        m = int(rng.integers(0, len(mats)))
        b = rng.uniform(-1, 1, mats[m][1].n_rows)
        prec = G.PRECISION_MIXED_F32 if k % 3 == 0 else G.PRECISION_F64
        reqs.append((m, b, prec))
    solver_id = {"cg": 0, "bicgstab": 1}

    def run(slots, together):
        S = G.Server(slots=slots)
        ids = [S.add_matrix(H) for H in handles]
        out = []
        if together:
            rids = [S.submit(ids[m], solver_id[mats[m][0]], b, 1e-10, 3000, G.opts(precision=p)) for m, b, p in reqs]
            out = [S.result(r) for r in rids]
        else:
            for m, b, p in reqs:
                out.append(S.result(S.submit(ids[m], solver_id[mats[m][0]], b, 1e-10, 3000, G.opts(precision=p))))
        st = S.stats()
        S.close()
        return out, st

    alone, st1 = run(1, False)
    mixed, st2 = run(6, True)
    assert st1["peak_active"] == 1 and st2["peak_active"] > 1
    assert st2["completed"] == len(reqs) and st2["p99_ms"] >= st2["p50_ms"] > 0
    for (s1, r1, x1, _), (s2, r2, x2, _), (m, b, p) in zip(alone, mixed, reqs):
        assert s1 == s2 == G.OK
        assert x1.tobytes() == x2.tobytes()
        assert r1.iterations == r2.iterations
        A = mats[m][1]
        assert np.linalg.norm(b - O.spmv_csr(A, x2)) <= 1.01e-10 * np.linalg.norm(b)


def test_budget_admission_and_rejections(gko):
    G = gko
    A = I.varcoef3d_7pt(40, np.random.default_rng(2))
    H = G.from_csr(A)
    mbytes = H.info()["bytes"]
    # budget for the matrix plus exactly one CG request (48 n bytes + 4 MiB)
    S = G.Server(slots=4, budget_bytes=mbytes + 48 * A.n_rows + (5 << 20))
    mid = S.add_matrix(H)
    b = np.random.default_rng(3).uniform(-1, 1, A.n_rows)
    rids = [S.submit(mid, 0, b, 1e-10, 3000) for _ in range(5)]
    res = [S.result(r) for r in rids]
    assert all(r[0] == G.OK for r in res)
    assert S.stats()["peak_active"] == 1
    with pytest.raises(G.GkoError) as e:
        S.submit(99, 0, b, 1e-10, 10)
    assert e.value.status == G.INVALID_ARG
    S.close()
    S = G.Server(slots=2, budget_bytes=mbytes + 1024)
    mid = S.add_matrix(H)
    with pytest.raises(G.GkoError) as e:
        S.submit(mid, 0, b, 1e-10, 10)
    assert e.value.status == G.BUDGET_EXCEEDED
    S.close()
    with pytest.raises(G.GkoError) as e:
        G.Server(slots=2, budget_bytes=1024).add_matrix(H)
    assert e.value.status == G.BUDGET_EXCEEDED


def test_nonblocking_poll(gko):
    G = gko
    A = I.varcoef3d_7pt(48, np.random.default_rng(4))
    S = G.Server(slots=2)
    mid = S.add_matrix(G.from_csr(A))
    rid = S.submit(mid, 0, np.ones(A.n_rows), 1e-12, 5000)
    first = S.result(rid, wait=False)
    final = first if first is not None else S.result(rid, wait=True)
    assert final[0] == G.OK and final[3] > 0
    S.close()


def test_bench_scale_mix_bitwise_alone(gko):
    """The serving benchmark's kind of load: 8 slots over resident matrices
    of sides 19..81 (Jacobi CG on variable-coefficient Poisson, BiCGSTAB on
    convection-diffusion), FP64 and mixed FP32, 160 requests queued at once.
    Every request must return GKO_OK with x bitwise equal to the same request
    solved alone on a one-slot server.  (Concurrent solves once summed stale
    bulk-copied SpMV stages here: 15-20% of the side-81 BiCGSTAB solves
    differed and some CG solves failed.)"""
    G = gko
    rng = np.random.default_rng(12)
    mats = [("cg", I.varcoef3d_7pt(side, rng)) for side in (72, 58, 35)]
    mats += [("bicgstab", I.convdiff3d_7pt(side, P)) for side, P in ((81, 8.0), (41, 3.0), (19, 12.0))]
    handles = [G.from_csr(A) for _, A in mats]
    bs = [O.spmv_csr(A, np.random.default_rng([3, m]).uniform(0.5, 1.5, A.n_rows)) for m, (_, A) in enumerate(mats)]
    arr = np.random.default_rng(13)
    reqs = [(int(arr.integers(0, 3)) if arr.random() < 0.7 else 3 + int(arr.integers(0, 3)),
             G.PRECISION_F64 if k % 2 == 0 else G.PRECISION_MIXED_F32) for k in range(160)]

    def opts(m, prec):
        if mats[m][0] == "cg":
            return G.opts(precision=prec, inner_maxit=1000, preconditioner=G.PRECOND_JACOBI)
        return G.opts(precision=prec, inner_maxit=1000)

    def submit(S, ids, m, prec):
        cg = mats[m][0] == "cg"
        return S.submit(ids[m], 0 if cg else 1, bs[m], 1e-8, 5000 if cg else 500, opts(m, prec))

    S = G.Server(slots=1)
    ids = [S.add_matrix(H) for H in handles]
    alone = {}
    for key in sorted(set(reqs)):
        alone[key] = S.result(submit(S, ids, *key))
    S.close()
    S = G.Server(slots=8, budget_bytes=150 << 30)
    ids = [S.add_matrix(H) for H in handles]
    rids = [submit(S, ids, m, prec) for m, prec in reqs]
    mixed = [S.result(r) for r in rids]
    st = S.stats()
    S.close()
    assert st["peak_active"] == 8
    bad = []
    for k, ((m, prec), (code, res, x, _)) in enumerate(zip(reqs, mixed)):
        c0, r0, x0, _ = alone[(m, prec)]
        assert c0 == G.OK, (m, prec, r0)
        if code != G.OK or x.tobytes() != x0.tobytes() or res.iterations != r0.iterations:
            bad.append((k, m, prec, code, res.iterations, r0.iterations))
    assert not bad, bad
    G.gko_device_status()
