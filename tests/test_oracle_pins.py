"""Pins for the CPU oracle: each check ties it to something other than itself.

* SpMV (all formats) against a dense brute-force product on integer data
  (exact in FP64), against closed-form Laplacian eigenpairs, and against
  exact rational sums (fractions) for the compensated variant.
* Conversions against an inverse written here (round trip to CSR) and the
  padding / nnz invariants of the Bell-Garland formats.
* The hybrid width rule against hand-derived cases (tests/golden).
* Solvers against dense LU solves (numpy), the exact solution of b = A*1, the
  n-step termination of CG and full GMRES, GMRES residual monotonicity and the
  FP32 accuracy floor of a single mixed-precision refinement step.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2006_14290_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U64 = 2.0**-53
U32 = 2.0**-24


def dense(A):
    D = np.zeros((A.n_rows, A.n_cols))
    for i in range(A.n_rows):
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            D[i, A.col[k]] += A.val[k]
    return D


# ------------------------------------------------------------------ SpMV --

@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (2.0, -3.0), (-1.0, 1.0), (0.0, 2.0)])
def test_spmv_csr_dense_bruteforce_integer_exact(seed, alpha, beta):
    rng = np.random.default_rng(seed)
    A = I.random_csr(37, 29, 0.25, rng, integer_values=True, empty_rows=0.2, sort_cols=False)
    x = rng.integers(-5, 6, 29).astype(float)
    y0 = rng.integers(-5, 6, 37).astype(float)
    y = O.spmv_csr(A, x, alpha, beta, y0)
    np.testing.assert_array_equal(y, alpha * (dense(A) @ x) + beta * y0)


def test_spmv_beta_zero_ignores_nan_in_y():
    rng = np.random.default_rng(3)
    A = I.random_csr(20, 20, 0.3, rng, integer_values=True)
    x = rng.integers(-3, 4, 20).astype(float)
    y0 = np.full(20, np.nan)
    y = O.spmv_csr(A, x, 1.5, 0.0, y0)
    assert np.all(np.isfinite(y))
    np.testing.assert_array_equal(y, 1.5 * (dense(A) @ x))


def test_spmv_nan_in_x_propagates_even_with_alpha_zero():
    A = I.laplace2d_5pt(4)
    x = np.ones(16)
    x[5] = np.nan
    y = O.spmv_csr(A, x, 0.0, 1.0, np.ones(16))
    rows_touching = {i for i in range(16) for k in range(A.row_ptr[i], A.row_ptr[i + 1]) if A.col[k] == 5}
    assert all(np.isnan(y[i]) for i in rows_touching)
    assert all(y[i] == 1.0 for i in range(16) if i not in rows_touching)


def _eig_check(A, v, lam):
    y = O.spmv_csr(A, v)
    normA = np.max(np.abs(A.val)) * np.max(np.diff(A.row_ptr))
    assert np.max(np.abs(y - lam * v)) <= 10 * U64 * normA * np.max(np.abs(v)) * 4


@pytest.mark.parametrize("N,p,q", [(6, 1, 1), (7, 2, 5), (9, 8, 3)])
def test_laplace2d_closed_form_eigenpairs(N, p, q):
    A = I.laplace2d_5pt(N)
    i = np.arange(N)
    sp_ = np.sin(p * math.pi * (i + 1) / (N + 1))
    sq = np.sin(q * math.pi * (i + 1) / (N + 1))
    v = (sp_[None, :] * sq[:, None]).reshape(-1)  # idx = i + N*j
    lam = 4 - 2 * math.cos(p * math.pi / (N + 1)) - 2 * math.cos(q * math.pi / (N + 1))
    _eig_check(A, v, lam)


@pytest.mark.parametrize("N,pqr", [(5, (1, 2, 3)), (6, (6, 1, 2))])
def test_stencil3d_7pt_closed_form_eigenpairs(N, pqr):
    A = I.stencil3d_7pt(N)
    i = np.arange(N)
    s = [np.sin(m * math.pi * (i + 1) / (N + 1)) for m in pqr]
    v = np.einsum("k,j,i->kji", s[2], s[1], s[0]).reshape(-1)
    lam = 6 - 2 * sum(math.cos(m * math.pi / (N + 1)) for m in pqr)
    _eig_check(A, v, lam)


@pytest.mark.parametrize("N,pqr", [(5, (1, 1, 1)), (6, (2, 5, 3))])
def test_stencil3d_27pt_closed_form_eigenpairs(N, pqr):
    # A = 27 I - T (x) T (x) T with T = tridiag(1, 1, 1); T's eigenvalues are
    # 1 + 2 cos(m pi / (N+1)) on the sine vectors.
    A = I.stencil3d_27pt(N)
    i = np.arange(N)
    s = [np.sin(m * math.pi * (i + 1) / (N + 1)) for m in pqr]
    v = np.einsum("k,j,i->kji", s[2], s[1], s[0]).reshape(-1)
    lam = 27 - np.prod([1 + 2 * math.cos(m * math.pi / (N + 1)) for m in pqr])
    _eig_check(A, v, lam)


def test_spmv_invariants_rowsums_and_columns():
    rng = np.random.default_rng(5)
    A = I.random_csr(40, 33, 0.2, rng, integer_values=True, sort_cols=False)
    D = dense(A)
    np.testing.assert_array_equal(O.spmv_csr(A, np.ones(33)), D.sum(axis=1))
    for j in (0, 7, 32):
        e = np.zeros(33)
        e[j] = 1.0
        np.testing.assert_array_equal(O.spmv_csr(A, e), D[:, j])


def test_spmv_exact_matches_rational_sum():
    rng = np.random.default_rng(7)
    lengths = [1, 5, 40, 200]
    A = I.rows_csr(lengths, 50, rng)
    # plant heavy cancellation: large +/- pairs
    A.val[5:7] = [1e16, -1e16]
    x = rng.uniform(-1, 1, 50)
    y = O.spmv_csr_exact(A, x)
    for i in range(len(lengths)):
        exact = sum((Fraction(float(A.val[k])) * Fraction(float(x[A.col[k]]))
                     for k in range(A.row_ptr[i], A.row_ptr[i + 1])), Fraction(0))
        assert abs(Fraction(float(y[i])) - exact) <= Fraction(2 * U64) * abs(exact) + Fraction(1e-300)


def test_spmv_f32_rounds_in_float_within_bound():
    rng = np.random.default_rng(11)
    A = I.rows_csr(rng.integers(1, 300, 200), 500, rng)
    x = rng.uniform(-1, 1, 500)
    x32 = x.astype(np.float32)
    y32 = O.spmv_csr_f32(A, x32)
    assert y32.dtype == np.float32
    A32 = I.Csr(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64))
    ex = O.spmv_csr_exact(A32, x32.astype(np.float64))
    s = O.spmv_abs_scale(A32, x32.astype(np.float64))
    lens = np.diff(A.row_ptr)
    err = np.abs(y32.astype(np.float64) - ex)
    assert np.all(err <= (lens + 2) * U32 * s)
    # and it is genuinely FP32: far from the FP64 sum on some rows
    assert np.max(err / np.maximum(s, 1e-300)) > 1e3 * U64


# ----------------------------------------------------------- conversions --

def _ell_to_csr(E, n):
    rows = []
    for i in range(n):
        cols, vals = [], []
        for k in range(E.K):
            c = E.col[k * E.stride + i]
            if c >= 0:
                cols.append(c)
                vals.append(E.val[k * E.stride + i])
        rows.append((cols, vals))
    return rows


def _csr_rows(A):
    return [(list(A.col[A.row_ptr[i]:A.row_ptr[i + 1]]), list(A.val[A.row_ptr[i]:A.row_ptr[i + 1]]))
            for i in range(A.n_rows)]


@pytest.mark.parametrize("seed", [0, 1])
def test_ell_round_trip_and_padding(seed):
    rng = np.random.default_rng(seed)
    A = I.random_csr(45, 60, 0.15, rng, empty_rows=0.2, sort_cols=False)
    E = O.csr_to_ell(A)
    assert E.stride == 64 and E.K == int(np.diff(A.row_ptr).max())
    assert _ell_to_csr(E, A.n_rows) == _csr_rows(A)
    pad = E.col < 0
    assert pad.sum() == E.K * E.stride - A.nnz
    assert np.all(E.col[pad] == -1) and np.all(E.val[pad] == 0.0)
    assert not np.any(np.signbit(E.val[pad]))
    x = rng.uniform(-1, 1, 60)
    np.testing.assert_array_equal(O.spmv_ell(E, x, 1.5, -0.5, np.ones(45)),
                                  O.spmv_csr(A, x, 1.5, -0.5, np.ones(45)))


def test_ell_padding_never_reads_x():
    A = I.rows_csr([1, 3, 0, 2], 4, np.random.default_rng(0))
    E = O.csr_to_ell(A)
    x = np.array([1.0, 2.0, 3.0, 4.0])
    used = set(A.col.tolist())
    for c in range(4):
        if c not in used:
            x[c] = np.inf
    assert np.all(np.isfinite(O.spmv_ell(E, x)))


def _sellp_to_csr(S):
    rows = []
    for i in range(S.n_rows):
        sl = i // S.C
        cols, vals = [], []
        for k in range(int(S.sets[sl + 1] - S.sets[sl])):
            q = (int(S.sets[sl]) + k) * S.C + i % S.C
            if S.col[q] >= 0:
                cols.append(int(S.col[q]))
                vals.append(float(S.val[q]))
        rows.append((cols, vals))
    return rows


def test_sellp_layout_golden():
    """A case laid out by hand from the SELL-P definition (C = 4)."""
    with open(os.path.join(GOLDEN, "sellp_layout_case.json")) as f:
        g = json.load(f)
    lens = [len(r[0]) for r in g["rows"]]
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    col = np.array([c for r in g["rows"] for c in r[0]], np.int32)
    val = np.array([v for r in g["rows"] for v in r[1]], np.float64)
    A = I.Csr(g["n_rows"], g["n_cols"], rp, col, val)
    S = O.csr_to_sellp(A, C=g["C"])
    np.testing.assert_array_equal(S.sets, g["sets"])
    np.testing.assert_array_equal(S.col, g["col"])
    np.testing.assert_array_equal(S.val, g["val"])


@pytest.mark.parametrize("C", [4, 32, 64])
@pytest.mark.parametrize("seed", [0, 1])
def test_sellp_round_trip_dense_and_padding(C, seed):
    """Inverse written here recovers the CSR rows; integer SpMV equals the
    dense product exactly; padding slots are col -1 / +0.0 and a slice whose
    rows are all empty has width 0."""
    rng = np.random.default_rng(seed)
    L = rng.integers(0, 9, 150)
    L[64:128] = 0  # a whole empty slice at C = 64 and C = 32
    A = I.rows_csr(L, 70, rng)
    A.val[:] = rng.integers(-4, 5, A.nnz)
    S = O.csr_to_sellp(A, C=C)
    assert _sellp_to_csr(S) == _csr_rows(A)
    widths = np.diff(S.sets)
    if C in (32, 64):
        assert widths[64 // C] == 0
    pad = S.col < 0
    assert pad.sum() == S.sets[-1] * C - A.nnz
    assert np.all(S.val[pad] == 0.0) and not np.any(np.signbit(S.val[pad]))
    x = rng.integers(-3, 4, 70).astype(float)
    y0 = rng.integers(-3, 4, 150).astype(float)
    np.testing.assert_array_equal(O.spmv_sellp(S, x, 2.0, -1.0, y0), 2.0 * (dense(A) @ x) - y0)


def test_sellp_padding_never_reads_x():
    A = I.rows_csr([1, 3, 0, 2, 5], 6, np.random.default_rng(0))
    S = O.csr_to_sellp(A, C=4)
    x = np.arange(1.0, 7.0)
    for c in set(range(6)) - set(A.col.tolist()):
        x[c] = np.inf
    assert np.all(np.isfinite(O.spmv_sellp(S, x)))


@pytest.mark.parametrize("S", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("loops", [1, 2, 3])
def test_subwarp_reduce_closed_form(S, loops):
    """After one butterfly round every lane of a subwarp holds the subwarp
    sum; each further round multiplies it by S (integer data, exact)."""
    rng = np.random.default_rng(S * 10 + loops)
    d = rng.integers(-9, 10, 128).astype(float)
    out = O.subwarp_reduce(d, S, loops)
    sums = d.reshape(-1, S).sum(axis=1)
    np.testing.assert_array_equal(out.reshape(-1, S), np.repeat((sums * S ** (loops - 1))[:, None], S, axis=1))


def test_coo_round_trip_and_dense():
    rng = np.random.default_rng(4)
    A = I.random_csr(50, 50, 0.1, rng, integer_values=True, empty_rows=0.3, sort_cols=False)
    M = O.csr_to_coo(A)
    assert M.nnz == A.nnz
    assert np.all(np.diff(M.row) >= 0)
    counts = np.bincount(M.row, minlength=50)
    np.testing.assert_array_equal(np.concatenate([[0], np.cumsum(counts)]), A.row_ptr)
    np.testing.assert_array_equal(M.col, A.col)
    np.testing.assert_array_equal(M.val, A.val)
    x = rng.integers(-3, 4, 50).astype(float)
    y0 = rng.integers(-3, 4, 50).astype(float)
    np.testing.assert_array_equal(O.spmv_coo(M, x, 2.0, 3.0, y0), 2.0 * (dense(A) @ x) + 3.0 * y0)


def test_hybrid_width_golden():
    with open(os.path.join(GOLDEN, "hybrid_width_cases.json")) as f:
        cases = json.load(f)["cases"]
    rng = np.random.default_rng(0)
    for c in cases:
        lens = np.concatenate([np.full(cnt, int(L)) for L, cnt in c["lengths"].items()])
        lens = rng.permutation(lens)
        rp = np.zeros(lens.size + 1, np.int64)
        np.cumsum(lens, out=rp[1:])
        A = I.Csr(lens.size, 16, rp.astype(np.int32), np.zeros(int(rp[-1]), np.int32), np.zeros(int(rp[-1])))
        assert O.hybrid_width(A) == c["K"], c["name"]
    assert O.hybrid_width(I.laplace2d_5pt(64)) == 3


@pytest.mark.parametrize("K", [None, 0, 2, 7])
def test_hybrid_round_trip(K):
    rng = np.random.default_rng(9)
    A = I.rows_csr(rng.integers(0, 12, 70), 70, rng)
    H = O.csr_to_hybrid(A, K)
    Kused = O.hybrid_width(A) if K is None else K
    assert H.ell.K == Kused
    ell_rows = _ell_to_csr(H.ell, A.n_rows)
    rows = []
    for i in range(A.n_rows):
        sel = H.coo.row == i
        rows.append((ell_rows[i][0] + list(H.coo.col[sel]), ell_rows[i][1] + list(H.coo.val[sel])))
    assert rows == _csr_rows(A)
    assert np.sum(H.ell.col >= 0) + H.coo.nnz == A.nnz
    assert np.all(np.diff(H.coo.row) >= 0)
    x = rng.uniform(-1, 1, 70)
    np.testing.assert_array_equal(O.spmv_hybrid(H, x, 1.0, 2.0, np.ones(70)),
                                  O.spmv_csr(A, x, 1.0, 2.0, np.ones(70)))


def test_workload_counts_golden():
    with open(os.path.join(GOLDEN, "workload_counts.json")) as f:
        g = json.load(f)
    small = {"laplace2d_5pt": (I.laplace2d_5pt, 2), "stencil3d_7pt": (I.stencil3d_7pt, 3),
             "stencil3d_27pt": (I.stencil3d_27pt, 3)}
    for c in g["closed_forms"]:
        fam = c["family"]
        if fam in small:
            f, dim = small[fam]
            for N in (3, 5, 8):
                A = f(N)
                nnz = {"laplace2d_5pt": 5 * N * N - 4 * N, "stencil3d_7pt": 7 * N**3 - 6 * N**2,
                       "stencil3d_27pt": (3 * N - 2) ** 3}[fam]
                assert A.n_rows == N**dim and A.nnz == nnz
    A = I.laplace2d_5pt(64)
    assert (A.n_rows, A.nnz) == (4096, 20224)
    B = I.convdiff3d_7pt(10, 3.0)
    assert B.nnz == 7 * 1000 - 600
    for s in g["seeded"]:
        if s["family"] == "powerlaw":
            P = I.powerlaw(s["n"], s["seed"])
            L = P.row_lengths()
            assert (P.nnz, int((L == 10000).sum()), int((L > 1024).sum())) == (
                s["nnz"], s["rows_at_10000"], s["rows_over_1024"])
        else:
            sides = I.batch_sides(s["count"], seed=s["seed"])
            assert int((sides**2).sum()) == s["sum_n"]
            assert int((5 * sides**2 - 4 * sides).sum()) == s["sum_nnz"]


# --------------------------------------------------------------- solvers --

def _spd(n, seed):
    rng = np.random.default_rng(seed)
    B = I.random_csr(n, n, 0.2, rng)
    D = dense(B)
    D = D + D.T
    D += np.diag(np.abs(D).sum(axis=1) + 1.0)
    return _from_dense(D)


def _from_dense(D):
    n = D.shape[0]
    rp = [0]
    cols, vals = [], []
    for i in range(n):
        nz = np.flatnonzero(D[i])
        cols += nz.tolist()
        vals += D[i, nz].tolist()
        rp.append(len(cols))
    return I.Csr(n, n, np.array(rp, np.int32), np.array(cols, np.int32), np.array(vals))


@pytest.mark.parametrize("n,seed", [(8, 0), (20, 1), (32, 2)])
def test_cg_n_step_and_dense_solve(n, seed):
    A = _spd(n, seed)
    b = np.random.default_rng(seed + 100).uniform(-1, 1, n)
    x, r = O.cg(A, b, tol=1e-10, maxit=10 * n)
    assert r.status == O.STATUS_OK and r.iterations <= n
    xd = np.linalg.solve(dense(A), b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    assert r.rel_residual <= 1e-10


def test_cg_b_equals_A_ones():
    A = I.laplace2d_5pt(16)
    b = O.spmv_csr(A, np.ones(A.n_rows))
    x, r = O.cg(A, b, tol=1e-12, maxit=1000)
    assert r.status == 0 and np.max(np.abs(x - 1)) < 1e-9


def test_cg_breakdown_on_indefinite_and_zero_rhs():
    A = _from_dense(np.diag([1.0, -1.0]))
    x, r = O.cg(A, np.array([1.0, 1.0]), tol=1e-12, maxit=10)
    assert r.status == O.STATUS_BREAKDOWN
    x, r = O.cg(I.laplace2d_5pt(4), np.zeros(16), x0=np.ones(16))
    assert r.status == 0 and r.iterations == 0 and np.all(x == 0)


def test_cg_reports_not_converged():
    A = I.laplace2d_5pt(32)
    b = np.random.default_rng(0).uniform(-1, 1, A.n_rows)
    x, r = O.cg(A, b, tol=1e-12, maxit=5)
    assert r.status == O.STATUS_NOT_CONVERGED and r.iterations == 5 and r.rel_residual > 1e-6


@pytest.mark.parametrize("N,P", [(3, 10.0), (4, 1.0), (5, 20.0)])
def test_bicgstab_dense_and_exact_ones(N, P):
    A = I.convdiff3d_7pt(N, P)
    b = dense(A) @ np.ones(A.n_rows)
    x, r = O.bicgstab(A, b, tol=1e-12, maxit=2000)
    assert r.status == 0 and r.rel_residual <= 1e-12
    assert np.max(np.abs(x - 1)) < 1e-8
    b2 = np.random.default_rng(N).uniform(-1, 1, A.n_rows)
    x2, r2 = O.bicgstab(A, b2, tol=1e-12, maxit=2000)
    xd = np.linalg.solve(dense(A), b2)
    assert np.linalg.norm(x2 - xd) <= 1e-8 * np.linalg.norm(xd)


@pytest.mark.parametrize("N,P", [(3, 10.0), (4, 2.0)])
def test_gmres_full_terminates_in_n_steps_monotone(N, P):
    A = I.convdiff3d_7pt(N, P)
    n = A.n_rows
    b = np.random.default_rng(1).uniform(-1, 1, n)
    x, r, hist = O.gmres(A, b, tol=1e-11, maxit=4 * n, restart=n, history=True)
    assert r.status == 0 and r.iterations <= n
    assert np.all(np.diff(hist) <= 1e-14)
    xd = np.linalg.solve(dense(A), b)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_gmres_restarted_matches_dense():
    A = I.convdiff3d_7pt(5, 10.0)
    b = dense(A) @ np.ones(A.n_rows)
    x, r = O.gmres(A, b, tol=1e-12, maxit=3000, restart=10)
    assert r.status == 0 and r.outer_iterations >= 2 and np.max(np.abs(x - 1)) < 1e-8


def test_gmres_nonsymmetric_small_nonsingular():
    D = np.array([[2.0, 1.0, 0.0], [0.0, 3.0, -1.0], [4.0, 0.0, 1.0]])
    A = _from_dense(D)
    b = np.array([1.0, -2.0, 0.5])
    x, r = O.gmres(A, b, tol=1e-14, maxit=10, restart=3)
    np.testing.assert_allclose(x, np.linalg.solve(D, b), rtol=1e-12)


@pytest.mark.parametrize("solver", [O.CG, O.BICGSTAB, O.GMRES])
def test_ir_reaches_fp64_tolerance(solver):
    A = I.laplace2d_5pt(24) if solver == O.CG else I.convdiff3d_7pt(6, 10.0)
    b = dense(A) @ np.ones(A.n_rows)
    x, r = O.solve_ir(solver, A, b, tol=1e-12, inner_tol=1e-4, inner_maxit=2000)
    assert r.status == 0 and r.rel_residual <= 1e-12 and r.outer_iterations >= 2
    assert np.max(np.abs(x - 1)) < 1e-9


def test_ir_single_step_limited_by_fp32_storage():
    # with an unreachable inner tolerance one refinement step is still capped
    # near the FP32 unit roundoff: the inner solve really stores in FP32
    A = I.varcoef2d_5pt(20, np.random.default_rng(3))
    b = np.random.default_rng(4).uniform(-1, 1, A.n_rows)
    x, r = O.solve_ir(O.CG, A, b, tol=1e-14, max_outer=1, inner_tol=1e-14, inner_maxit=400)
    assert r.status == O.STATUS_NOT_CONVERGED
    assert 1e-9 < r.rel_residual < 1e-4
    x2, r2 = O.solve_ir(O.CG, A, b, tol=1e-12, max_outer=30, inner_tol=1e-5, inner_maxit=400)
    assert r2.status == 0 and r2.rel_residual <= 1e-12


def test_ir_inner_update_is_fp32_stored():
    # from x0 = 0 one refinement step sets x = d, and d is stored in FP32
    A = I.laplace2d_5pt(12)
    b = np.random.default_rng(8).uniform(-1, 1, A.n_rows)
    x, r = O.solve_ir(O.CG, A, b, tol=1e-14, max_outer=1, inner_tol=1e-3, inner_maxit=100)
    assert r.outer_iterations == 1
    np.testing.assert_array_equal(x.astype(np.float32).astype(np.float64), x)
    for solver in (O.BICGSTAB, O.GMRES):
        B = I.convdiff3d_7pt(4, 5.0)
        bb = np.random.default_rng(9).uniform(-1, 1, B.n_rows)
        x, r = O.solve_ir(solver, B, bb, tol=1e-14, max_outer=1, inner_tol=1e-3, inner_maxit=100)
        np.testing.assert_array_equal(x.astype(np.float32).astype(np.float64), x)


# ---------------------------------------------------------------- BLAS-1 --

def test_blas1_exact_on_integers_and_rationals():
    rng = np.random.default_rng(12)
    x = rng.integers(-9, 10, 300).astype(float)
    y = rng.integers(-9, 10, 300).astype(float)
    assert O.dot(x, y) == float(sum(int(a) * int(b) for a, b in zip(x, y)))
    np.testing.assert_array_equal(O.axpy(-3.0, x, y), -3.0 * x + y)
    V = rng.integers(-3, 4, (5, 300)).astype(float)
    h = O.multi_dot(V, x)
    np.testing.assert_array_equal(h, [sum(int(a) * int(b) for a, b in zip(v, x)) for v in V])
    hh = rng.integers(-2, 3, 5).astype(float)
    out, nrm = O.multi_axpy_norm(V, hh, y)
    ref = y - hh @ V
    np.testing.assert_array_equal(out, ref)
    assert nrm == pytest.approx(math.sqrt(float(sum(int(v) ** 2 for v in ref))), rel=1e-15)
    # rational check of a non-integer dot
    xf = rng.uniform(-1, 1, 50)
    yf = rng.uniform(-1, 1, 50)
    ex = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(xf, yf))
    bound = 50 * U64 * float(sum(abs(Fraction(float(a)) * Fraction(float(b))) for a, b in zip(xf, yf)))
    assert abs(O.dot(xf, yf) - float(ex)) <= bound


# -------------------------------------------------------------- Jacobi --

def test_jacobi_inv_sums_diagonal_duplicates_and_guards_zero():
    A = I.Csr(3, 3, np.array([0, 3, 3, 5], np.int32), np.array([0, 1, 0, 2, 2], np.int32),
              np.array([2.0, 7.0, 2.0, 1.0, 3.0]))
    np.testing.assert_array_equal(O.jacobi_inv(A), [0.25, 1.0, 0.25])


def test_pcg_on_diagonal_matrix_is_exact_in_one_step():
    d = np.array([1.0, 4.0, 0.5, 8.0, 2.0])
    A = I.rows_csr([1] * 5, 5, np.random.default_rng(0))
    A.col[:] = np.arange(5)
    A.val[:] = d
    b = np.array([3.0, 1.0, -2.0, 4.0, 0.5])
    x, r = O.solve_jacobi(O.CG, A, b, tol=1e-14, maxit=10)
    assert r.status == 0 and r.iterations == 1
    np.testing.assert_allclose(x, b / d, rtol=1e-15)


def test_pcg_equals_cg_for_constant_diagonal():
    """M = 6 I: z = r/6 is a uniform rescaling, so PCG runs CG's iterates."""
    A = I.stencil3d_7pt(6)
    b = dense(A) @ np.ones(A.n_rows)
    x1, r1 = O.cg(A, b, tol=1e-12, maxit=500)
    x2, r2 = O.solve_jacobi(O.CG, A, b, tol=1e-12, maxit=500)
    assert r1.iterations == r2.iterations
    np.testing.assert_allclose(x2, x1, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("solver", ["cg", "bicgstab"])
def test_jacobi_solves_badly_scaled_systems(solver):
    """D A D with a wide diagonal scaling D: the Jacobi-preconditioned solve
    matches a dense solve and needs far fewer iterations than without."""
    rng = np.random.default_rng(3)
    A = I.laplace2d_5pt(12) if solver == "cg" else I.convdiff3d_7pt(5, 2.0)
    n = A.n_rows
    s = np.exp(rng.uniform(-3, 3, n))
    rows = np.repeat(np.arange(n), np.diff(A.row_ptr))
    A.val[:] = A.val * s[rows] * s[A.col]
    b = rng.uniform(-1, 1, n)
    xd = np.linalg.solve(dense(A), b)
    which = O.CG if solver == "cg" else O.BICGSTAB
    x0, r0 = O.solve(which, A, b, tol=1e-10, maxit=20000)
    x1, r1 = O.solve_jacobi(which, A, b, tol=1e-10, maxit=20000)
    assert r1.status == 0 and r1.rel_residual <= 1e-10
    assert np.linalg.norm(x1 - xd) <= 1e-6 * np.linalg.norm(xd)
    assert r1.iterations < 0.5 * r0.iterations, (r1.iterations, r0.iterations)


def test_jacobi_ir_reaches_fp64_tolerance():
    rng = np.random.default_rng(5)
    A = I.varcoef3d_7pt(8, rng)
    b = dense(A) @ np.ones(A.n_rows)
    x, r = O.solve_ir(O.CG, A, b, tol=1e-10, inner_tol=1e-5, jacobi=True)
    assert r.status == 0 and r.rel_residual <= 1e-10 and r.outer_iterations >= 2
    np.testing.assert_allclose(x, np.ones(A.n_rows), rtol=1e-7)


def test_jacobi_gmres_refused():
    A = I.laplace2d_5pt(4)
    x, r = O.solve_jacobi(O.GMRES, A, np.ones(16))
    assert r.status == 1


# -------------------------------------------------------- block-Jacobi --

def csr_from_dense(D, dup=None):
    """CSR of a dense matrix (nonzeros in ascending column order); dup =
    (i, j, v) splits entry (i, j) into v and D[i, j] - v stored twice."""
    rp, col, val = [0], [], []
    for i in range(D.shape[0]):
        for j in range(D.shape[1]):
            if D[i, j] != 0.0:
                if dup is not None and (i, j) == dup[:2]:
                    col += [j, j]
                    val += [dup[2], D[i, j] - dup[2]]
                else:
                    col.append(j)
                    val.append(D[i, j])
        rp.append(len(col))
    return I.Csr(D.shape[0], D.shape[1], np.array(rp, np.int32), np.array(col, np.int32),
                 np.array(val, np.float64))


@pytest.mark.parametrize("n,bs", [(37, 8), (32, 4), (5, 8), (40, 1), (33, 32)])
def test_block_jacobi_inverts_each_diagonal_block(n, bs):
    """Each block of B is the inverse of the matching diagonal block of A
    (numpy's LU-based inverse and B D = I), off-block entries play no part,
    and the last block of n % bs rows is inverted on its own."""
    rng = np.random.default_rng(n * 100 + bs)
    D = rng.uniform(-1, 1, (n, n)) * (rng.uniform(0, 1, (n, n)) < 0.5)
    D += np.diag(rng.uniform(2, 4, n) * rng.choice([-1, 1], n))  # nonsymmetric, nonsingular blocks
    B, singular = O.block_jacobi_inv(csr_from_dense(D), bs)
    assert singular == 0 and B.shape == (n, bs)
    for base in range(0, n, bs):
        nb = min(bs, n - base)
        blk = D[base:base + nb, base:base + nb]
        inv = B[base:base + nb, :nb]
        np.testing.assert_allclose(inv, np.linalg.inv(blk), rtol=0, atol=1e-13 * np.linalg.cond(blk))
        np.testing.assert_allclose(inv @ blk, np.eye(nb), rtol=0, atol=1e-13 * np.linalg.cond(blk))
        assert np.all(B[base:base + nb, nb:] == 0.0)


def test_block_jacobi_pivots_sums_duplicates_and_replaces_singular_blocks():
    # block 0 = [[0, 2], [3, 1]] needs a row swap; its inverse is
    # [[-1/6, 1/3], [1/2, 0]].  Block 1 = [[1, 2], [2, 4]] is singular and
    # becomes the identity; block 2 is the single row 5 (stored as 1.5 + 3.5).
    D = np.zeros((5, 5))
    D[0, 1], D[1, 0], D[1, 1] = 2.0, 3.0, 1.0
    D[2, 2], D[2, 3], D[3, 2], D[3, 3] = 1.0, 2.0, 2.0, 4.0
    D[4, 4] = 5.0
    D[0, 4], D[4, 0] = 7.0, -9.0  # outside every block
    B, singular = O.block_jacobi_inv(csr_from_dense(D, dup=(4, 4, 1.5)), 2)
    assert singular == 1
    exact = [[Fraction(-1, 6), Fraction(1, 3)], [Fraction(1, 2), Fraction(0)]]
    for i in range(2):
        for j in range(2):
            assert abs(B[i, j] - float(exact[i][j])) <= 2 * U64 * abs(float(exact[i][j]))
    np.testing.assert_array_equal(B[2:4], np.eye(2))
    np.testing.assert_array_equal(B[4], [0.2, 0.0])


def test_block_jacobi_block_size_one_is_jacobi():
    rng = np.random.default_rng(7)
    A = I.varcoef3d_7pt(5, rng)
    Z = I.Csr(A.n_rows, A.n_cols, A.row_ptr.copy(), A.col.copy(), A.val.copy())
    diag = np.flatnonzero(Z.col == np.repeat(np.arange(Z.n_rows), np.diff(Z.row_ptr)))
    Z.val[diag[3]] = 0.0  # a zero diagonal: Jacobi takes 1, block size 1 the identity block
    B, singular = O.block_jacobi_inv(Z, 1)
    assert singular == 1
    np.testing.assert_array_equal(B[:, 0], O.jacobi_inv(Z))
    b = rng.uniform(-1, 1, A.n_rows)
    for solver in (O.CG, O.BICGSTAB):
        x1, r1 = O.solve_jacobi(solver, A, b, tol=1e-10, maxit=2000)
        x2, r2 = O.solve_block_jacobi(solver, A, b, 1, tol=1e-10, maxit=2000)
        assert r1.iterations == r2.iterations
        np.testing.assert_array_equal(x1, x2)


@pytest.mark.parametrize("solver", ["cg", "bicgstab"])
def test_block_jacobi_exact_on_block_diagonal_matrix(solver):
    """A block diagonal with blocks of bs rows: M = A, so the preconditioned
    operator is the identity and one iteration solves the system."""
    rng = np.random.default_rng(11)
    n, bs = 29, 4
    D = np.zeros((n, n))
    for base in range(0, n, bs):
        nb = min(bs, n - base)
        Q = rng.uniform(-1, 1, (nb, nb))
        D[base:base + nb, base:base + nb] = Q @ Q.T + nb * np.eye(nb) if solver == "cg" else Q + 3 * np.eye(nb)
    b = rng.uniform(-1, 1, n)
    which = O.CG if solver == "cg" else O.BICGSTAB
    x, r = O.solve_block_jacobi(which, csr_from_dense(D), b, bs, tol=1e-12, maxit=10)
    assert r.status == 0 and r.iterations == 1
    np.testing.assert_allclose(x, np.linalg.solve(D, b), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("solver,bs", [("cg", 4), ("cg", 8), ("bicgstab", 2), ("bicgstab", 16)])
def test_block_jacobi_solves_badly_scaled_systems(solver, bs):
    """Rows and columns scaled blockwise by D A D with a wide scaling: the
    block-Jacobi solve matches a dense solve and needs fewer iterations
    than the unpreconditioned one."""
    rng = np.random.default_rng(13)
    A = I.laplace2d_5pt(11) if solver == "cg" else I.convdiff3d_7pt(5, 2.0)
    n = A.n_rows
    sc = np.exp(rng.uniform(-3, 3, n))
    rows = np.repeat(np.arange(n), np.diff(A.row_ptr))
    A.val[:] = A.val * sc[rows] * sc[A.col]
    b = rng.uniform(-1, 1, n)
    xd = np.linalg.solve(dense(A), b)
    which = O.CG if solver == "cg" else O.BICGSTAB
    x0, r0 = O.solve(which, A, b, tol=1e-10, maxit=20000)
    x1, r1 = O.solve_block_jacobi(which, A, b, bs, tol=1e-10, maxit=20000)
    assert r1.status == 0 and r1.rel_residual <= 1e-10
    assert np.linalg.norm(x1 - xd) <= 1e-6 * np.linalg.norm(xd)
    assert r1.iterations < 0.5 * r0.iterations, (r1.iterations, r0.iterations)


@pytest.mark.parametrize("solver", ["cg", "bicgstab"])
def test_block_jacobi_mixed_size_one_is_mixed_jacobi(solver):
    """With blocks of one row the FP32-rounded inverse blocks are the FP32
    Jacobi inverse, so the mixed solves (restarted refinement and reliable
    updates) repeat the Jacobi ones bit for bit."""
    rng = np.random.default_rng(17)
    A = I.varcoef3d_7pt(6, rng) if solver == "cg" else I.convdiff3d_7pt(6, 2.0)
    b = rng.uniform(-1, 1, A.n_rows)
    which = O.CG if solver == "cg" else O.BICGSTAB
    x1, r1 = O.solve_ir(which, A, b, tol=1e-10, inner_tol=1e-5, jacobi=True)
    x2, r2 = O.solve_ir(which, A, b, tol=1e-10, inner_tol=1e-5, block_size=1)
    assert (r1.iterations, r1.outer_iterations) == (r2.iterations, r2.outer_iterations)
    np.testing.assert_array_equal(x1, x2)
    x1, r1 = O.solve_reliable(which, A, b, tol=1e-12, jacobi=True)
    x2, r2 = O.solve_reliable(which, A, b, tol=1e-12, block_size=1)
    assert (r1.iterations, r1.outer_iterations) == (r2.iterations, r2.outer_iterations)
    np.testing.assert_array_equal(x1, x2)


@pytest.mark.parametrize("solver,bs", [("cg", 4), ("cg", 16), ("bicgstab", 8)])
def test_block_jacobi_mixed_reaches_fp64_accuracy(solver, bs):
    """FP32 recurrences preconditioned by FP32-rounded inverse blocks: the
    FP64 refinement (restarted, and by reliable updates) still reaches FP64
    tolerances and the dense solution; the reliable-update solve with the FP64
    operator, FP64 storage and delta = 0 is the FP64 block-Jacobi solve."""
    rng = np.random.default_rng(19)
    A = scaled_copy(I.laplace2d_5pt(13) if solver == "cg" else I.convdiff3d_7pt(6, 2.0), rng)
    b = rng.uniform(-1, 1, A.n_rows)
    xd = np.linalg.solve(dense(A), b)
    which = O.CG if solver == "cg" else O.BICGSTAB
    x, r = O.solve_ir(which, A, b, tol=1e-10, inner_tol=1e-5, inner_maxit=5000, block_size=bs)
    assert r.status == 0 and r.rel_residual <= 1e-10 and r.outer_iterations >= 2
    assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)
    x, r = O.solve_reliable(which, A, b, tol=1e-12, maxit=5000, block_size=bs)
    assert r.status == 0 and r.rel_residual <= 1e-12 and r.outer_iterations >= 1
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    x1, r1 = O.solve_reliable(which, A, b, tol=1e-10, maxit=5000, delta=0.0, f32=False, block_size=bs)
    x2, r2 = O.solve_block_jacobi(which, A, b, bs, tol=1e-10, maxit=5000)
    assert r1.iterations == r2.iterations
    np.testing.assert_array_equal(x1, x2)


def scaled_copy(A, rng, spread=2.0):
    s = np.exp(rng.uniform(-spread, spread, A.n_rows))
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    return I.Csr(A.n_rows, A.n_cols, A.row_ptr.copy(), A.col.copy(), A.val * s[rows] * s[A.col])


def test_block_jacobi_gmres_and_bad_block_size_refused():
    A = I.laplace2d_5pt(4)
    x, r = O.solve_block_jacobi(O.GMRES, A, np.ones(16), 4)
    assert r.status == 1
    with pytest.raises(ValueError):
        O.block_jacobi_inv(A, 0)


def test_batch_cg_is_the_single_system_cg_per_system():
    """The batched oracle (c8: CG applied to each system on its own) equals
    the single-system CG bit for bit, whatever the thread count, and its
    solutions agree with dense solves."""
    sides = [5, 8, 3, 11, 6]
    systems, bs = [], []
    for i, sd in enumerate(sides):
        A, b = I.batch_system(i, sd)
        systems.append(A)
        bs.append(b)
    bs[2] = np.zeros_like(bs[2])
    outs = []
    for threads in (1, 4):
        O.set_threads(threads)
        outs.append(O.batch_cg(systems, bs, tol=1e-12, maxit=5000))
    O.set_threads(1)
    (x1, it1, rr1, st1), (x4, it4, rr4, st4) = outs
    for i, (A, b) in enumerate(zip(systems, bs)):
        xs, rs = O.cg(A, b, tol=1e-12, maxit=5000)
        assert x1[i].tobytes() == xs.tobytes() == x4[i].tobytes()
        assert it1[i] == rs.iterations == it4[i] and st1[i] == rs.status == 0
        assert rr1[i] == rs.rel_residual
        if i != 2:
            D = np.zeros((A.n_rows, A.n_rows))
            for r in range(A.n_rows):
                D[r, A.col[A.row_ptr[r]:A.row_ptr[r + 1]]] += A.val[A.row_ptr[r]:A.row_ptr[r + 1]]
            xd = np.linalg.solve(D, b)
            assert np.linalg.norm(xs - xd) <= 1e-9 * np.linalg.norm(xd)
        else:
            assert np.all(x1[i] == 0) and it1[i] == 0


def test_ir_fixed_inner_tolerance_contracts_by_inner_tol():
    """With the inner solve held to a fixed relative tolerance, each
    refinement step reduces the true residual by about inner_tol (the FP32
    storage floor is far below 1e-4 here): 1e-12 takes exactly 3 steps at
    inner_tol 1e-4 and 4 at 1e-3 (reductions compound as inner_tol^k).  The
    library's adaptive tunable needs no more steps."""
    A = I.laplace2d_5pt(24)
    b = dense(A) @ np.ones(A.n_rows)
    _, r4 = O.solve_ir(O.CG, A, b, tol=1e-12, inner_tol=1e-4, inner_maxit=2000)
    _, r3 = O.solve_ir(O.CG, A, b, tol=1e-12, inner_tol=1e-3, inner_maxit=2000)
    _, ra = O.solve_ir(O.CG, A, b, tol=1e-12, inner_tol=1e-4, inner_maxit=2000, adaptive=True)
    assert r4.status == r3.status == ra.status == 0
    assert r4.outer_iterations == 3 and r3.outer_iterations == 4, (r4, r3)
    assert ra.outer_iterations <= r4.outer_iterations


# ------------------------------------------------- reliable-update solves --

@pytest.mark.parametrize("solver", [O.CG, O.BICGSTAB])
@pytest.mark.parametrize("N", [4, 8, 12])
def test_reliable_fp64_without_updates_is_the_plain_solver(solver, N):
    # FP64 operator and storage, delta = 0: the only update is the final check,
    # and with x0 = 0 the folded partial solution is the plain solver's iterate,
    # so iterations and x agree bit for bit with textbook CG / BiCGSTAB (pinned
    # above against dense solves)
    A = I.stencil3d_7pt(N) if solver == O.CG else I.convdiff3d_7pt(N, 3.0)
    b = np.random.default_rng(N).uniform(-1, 1, A.n_rows)
    x0, r0 = O.solve(solver, A, b, tol=1e-11, maxit=5000)
    x1, r1 = O.solve_reliable(solver, A, b, tol=1e-11, maxit=5000, delta=0.0, f32=False)
    assert r0.status == r1.status == 0
    assert r1.iterations == r0.iterations and r1.outer_iterations == 1
    np.testing.assert_array_equal(x1, x0)


@pytest.mark.parametrize("solver,N,P", [(O.CG, 8, 0.0), (O.BICGSTAB, 8, 1.0), (O.BICGSTAB, 7, 10.0)])
def test_reliable_mixed_reaches_fp64_accuracy(solver, N, P):
    # FP32 values and vectors in the recurrences: the FP64 replacements still
    # bring the true residual to 1e-12, and x agrees with a dense solve
    A = I.varcoef3d_7pt(N, np.random.default_rng(2)) if solver == O.CG else I.convdiff3d_7pt(N, P)
    b = np.random.default_rng(5).uniform(-1, 1, A.n_rows)
    x, r = O.solve_reliable(solver, A, b, tol=1e-12, maxit=5000, delta=0.1)
    assert r.status == 0 and r.rel_residual <= 1e-12 and r.outer_iterations >= 3
    D = dense(A)
    xd = np.linalg.solve(D, b)
    kappa = np.linalg.cond(D)
    assert np.linalg.norm(x - xd) <= 10 * kappa * 1e-12 * np.linalg.norm(xd)


def test_reliable_recurrences_are_fp32_and_updates_matter():
    # the recurrences really run in FP32: with updates only when the FP32
    # recurrence residual meets the tolerance (delta = 0), the true residual
    # stalls far above 1e-12; the delta updates bring it there
    A = I.varcoef2d_5pt(24, np.random.default_rng(3))
    b = np.random.default_rng(4).uniform(-1, 1, A.n_rows)
    x, r = O.solve_reliable(O.CG, A, b, tol=1e-12, maxit=3000, delta=0.0)
    assert r.status == O.STATUS_NOT_CONVERGED and r.rel_residual > 1e-9
    x, r = O.solve_reliable(O.CG, A, b, tol=1e-12, maxit=3000, delta=0.1)
    assert r.status == 0 and r.rel_residual <= 1e-12 and r.outer_iterations >= 3
    xd = np.linalg.solve(dense(A), b)
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_reliable_jacobi_zero_rhs_and_x0():
    A = I.varcoef3d_7pt(6, np.random.default_rng(7))
    b = np.random.default_rng(8).uniform(-1, 1, A.n_rows)
    xd = np.linalg.solve(dense(A), b)
    for solver in (O.CG, O.BICGSTAB):
        x, r = O.solve_reliable(solver, A, b, tol=1e-12, maxit=5000, delta=0.1, jacobi=True)
        assert r.status == 0 and np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
        x, r = O.solve_reliable(solver, A, np.zeros(A.n_rows), x0=np.ones(A.n_rows))
        assert r.status == 0 and r.iterations == 0 and np.all(x == 0)
        x, r = O.solve_reliable(solver, A, b, x0=xd, tol=1e-8)
        assert r.status == 0 and r.iterations == 0 and r.outer_iterations == 0
    x, r = O.solve_reliable(O.CG, A, b, tol=1e-12, maxit=3)
    assert r.status == O.STATUS_NOT_CONVERGED and r.iterations == 3


@pytest.mark.parametrize("solver", [O.CG, O.BICGSTAB])
def test_reliable_partial_solution_is_fp32_stored(solver):
    # from x0 = 0 with no update before the iteration cap, x is the folded
    # partial solution y, which the recurrences store in FP32
    A = I.laplace2d_5pt(12) if solver == O.CG else I.convdiff3d_7pt(5, 5.0)
    b = np.random.default_rng(11).uniform(-1, 1, A.n_rows)
    x, r = O.solve_reliable(solver, A, b, tol=1e-14, maxit=4, delta=0.0)
    assert r.status == O.STATUS_NOT_CONVERGED and r.outer_iterations == 0
    np.testing.assert_array_equal(x.astype(np.float32).astype(np.float64), x)
    assert np.any(x != 0)


def test_batch_cg_reliable_is_the_single_system_solve_per_system():
    """The batched reliable-update oracle equals the single-system
    reliable-update CG bit for bit whatever the thread count, reaches the
    tolerance in FP64 and agrees with dense solves; with FP32 storage the
    systems are the FP32-rounded ones."""
    sides = [5, 9, 3, 12, 7]
    systems, bs = [], []
    for i, sd in enumerate(sides):
        A, b = I.batch_system(i, sd)
        systems.append(A)
        bs.append(b)
    bs[2] = np.zeros_like(bs[2])
    outs = []
    for threads in (1, 4):
        O.set_threads(threads)
        outs.append(O.batch_cg_reliable(systems, bs, tol=1e-12, maxit=5000))
    O.set_threads(1)
    (x1, it1, up1, rr1, st1), (x4, it4, up4, rr4, st4) = outs
    for i, (A, b) in enumerate(zip(systems, bs)):
        xs, rs = O.solve_reliable(O.CG, A, b, tol=1e-12, maxit=5000, delta=0.1)
        assert x1[i].tobytes() == xs.tobytes() == x4[i].tobytes()
        assert it1[i] == rs.iterations == it4[i] and up1[i] == rs.outer_iterations == up4[i]
        assert st1[i] == rs.status == 0 and rr1[i] == rs.rel_residual
        if i != 2:
            assert rr1[i] <= 1e-12
            xd = np.linalg.solve(dense(A), b)
            assert np.linalg.norm(xs - xd) <= 1e-8 * np.linalg.norm(xd)
        else:
            assert np.all(x1[i] == 0) and it1[i] == 0
    x32, it32, up32, rr32, st32 = O.batch_cg_reliable(systems, bs, tol=1e-12, maxit=5000, storage_f32=True)
    for i, (A, b) in enumerate(zip(systems, bs)):
        if i == 2:
            continue
        A32 = I.Csr(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64))
        assert st32[i] == 0 and np.linalg.norm(b - dense(A32) @ x32[i]) <= 1.01e-12 * np.linalg.norm(b)
