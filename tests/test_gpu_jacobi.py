"""GPU parity of Jacobi-preconditioned CG and right-preconditioned BiCGSTAB
(FP64 and inside mixed-precision refinement) against the CPU oracle, on
badly scaled systems in every format, through the C ABI."""
import numpy as np
import pytest

import oracle as O
from gpu_util import dev, host
from paper_2006_14290_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def scaled(A, seed=3, spread=3.0):
    """D A D with log-uniform D in [e^-spread, e^spread]: Jacobi's home turf."""
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(-spread, spread, A.n_rows))
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    A.val[:] = A.val * s[rows] * s[A.col]
    return A


def convert(G, M, fmt):
    if fmt == "ell":
        return G.gko_matrix_convert_to_ell(M)
    if fmt == "coo":
        return G.gko_matrix_convert_to_coo(M)
    if fmt == "hybrid":
        return G.gko_matrix_convert_to_hybrid(M, 3)
    if fmt == "sellp":
        return G.gko_matrix_convert_to_sellp(M, 32)
    return M


def solve(G, name, M, b, tol, maxit, **opt):
    xd = dev(np.zeros(b.size))
    fn = G.gko_solve_cg if name == "cg" else G.gko_solve_bicgstab
    res = fn(M, dev(b), xd, tol, maxit, G.opts(**opt))
    return host(xd), res


def iters_close(a, b):
    return abs(a - b) <= max(2, 0.1 * max(a, b))


@pytest.mark.parametrize("fmt", ["csr", "ell", "coo", "hybrid", "sellp"])
@pytest.mark.parametrize("name", ["cg", "bicgstab"])
def test_jacobi_matches_oracle(gko, fmt, name):
    G = gko
    A = scaled(I.laplace2d_5pt(40) if name == "cg" else I.convdiff3d_7pt(10, 3.0))
    b = np.random.default_rng(9).uniform(-1, 1, A.n_rows)
    M = convert(G, G.from_csr(A), fmt)
    which = O.CG if name == "cg" else O.BICGSTAB
    xo, ro = O.solve_jacobi(which, A, b, tol=1e-12, maxit=20000)
    xg, rg = solve(G, name, M, b, 1e-12, 20000, preconditioner=G.PRECOND_JACOBI)
    assert ro.status == 0 and rg.status == G.OK, (ro, rg)
    assert rg.rel_residual <= 1e-12
    assert np.linalg.norm(b - O.spmv_csr(A, xg)) <= 1.01e-12 * np.linalg.norm(b)
    assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)
    assert iters_close(rg.iterations, ro.iterations), (rg.iterations, ro.iterations)
    _, r0 = solve(G, name, M, b, 1e-12, 20000)  # unpreconditioned: many more iterations here
    assert rg.iterations < 0.5 * r0.iterations, (rg.iterations, r0.iterations)


@pytest.mark.parametrize("name", ["cg", "bicgstab"])
def test_jacobi_mixed_precision_matches_oracle(gko, name):
    G = gko
    A = scaled(I.laplace2d_5pt(40) if name == "cg" else I.convdiff3d_7pt(10, 3.0), spread=2.0)
    b = O.spmv_csr(A, np.ones(A.n_rows))
    M = G.from_csr(A)
    which = O.CG if name == "cg" else O.BICGSTAB
    xo, ro = O.solve_ir(which, A, b, tol=1e-10, inner_tol=1e-5, inner_maxit=5000, jacobi=True, adaptive=True)
    xg, rg = solve(G, name, M, b, 1e-10, 5000, precision=G.PRECISION_MIXED_F32, inner_tol=1e-5,
                   inner_maxit=5000, preconditioner=G.PRECOND_JACOBI, refinement=G.REFINE_RESTART)
    assert ro.status == 0 and rg.status == G.OK, (ro, rg)
    assert rg.rel_residual <= 1e-10
    assert np.linalg.norm(xg - np.ones(A.n_rows)) <= 1e-6 * np.sqrt(A.n_rows)
    assert abs(rg.outer_iterations - ro.outer_iterations) <= 1
    # reliable updates (FP32 recurrences, FP64 replacements) with Jacobi
    xr, rr = O.solve_reliable(which, A, b, tol=1e-12, maxit=5000, delta=0.1, jacobi=True)
    xg, rg = solve(G, name, M, b, 1e-12, 5000, precision=G.PRECISION_MIXED_F32, preconditioner=G.PRECOND_JACOBI,
                   refinement=G.REFINE_RELIABLE)
    assert rr.status == 0 and rg.status == G.OK, (rr, rg)
    assert np.linalg.norm(b - O.spmv_csr(A, xg)) <= 1.01e-12 * np.linalg.norm(b)
    assert np.linalg.norm(xg - xr) <= 1e-8 * np.linalg.norm(xr)


@pytest.mark.parametrize("fmt", ["csr", "ell", "coo", "hybrid", "sellp"])
def test_jacobi_diagonal_system_one_step(gko, fmt):
    """A diagonal matrix stored with each diagonal value split into two
    duplicate entries (for hybrid width 1 one lands in the ELL part and one
    in the COO tail): the inverse diagonal must sum them, and one
    preconditioned CG step is then exact."""
    G = gko
    n = 300
    d = np.exp(np.random.default_rng(2).uniform(-2, 2, n))
    rp = np.arange(0, 2 * n + 1, 2, dtype=np.int32)
    col = np.repeat(np.arange(n, dtype=np.int32), 2)
    val = np.repeat(d / 2, 2)
    val[1::2] = d - val[0::2]
    A = I.Csr(n, n, rp, col, val)
    M = G.from_csr(A)
    M = G.gko_matrix_convert_to_hybrid(M, 1) if fmt == "hybrid" else convert(G, M, fmt)
    b = np.random.default_rng(4).uniform(-1, 1, n)
    xg, rg = solve(G, "cg", M, b, 1e-13, 10, preconditioner=G.PRECOND_JACOBI)
    assert rg.status == G.OK and rg.iterations == 1
    np.testing.assert_allclose(xg, b / (val[0::2] + val[1::2]), rtol=1e-14)


def test_jacobi_refusals(gko):
    G = gko
    A = I.laplace2d_5pt(8)
    M = G.from_csr(A)
    b = dev(np.ones(A.n_rows))
    with pytest.raises(G.GkoError) as e:
        G.gko_solve_gmres(M, b, dev(np.zeros(A.n_rows)), 1e-8, 100, G.opts(preconditioner=G.PRECOND_JACOBI))
    assert e.value.status == G.NOT_SUPPORTED
    with pytest.raises(G.GkoError) as e:
        G.gko_solve_cg(M, b, dev(np.zeros(A.n_rows)), 1e-8, 100, G.opts(preconditioner=7))
    assert e.value.status == G.INVALID_ARG


@pytest.mark.parametrize("N", [16, 17, 20, 24])
def test_small_mixed_jacobi_inner_solve_matches_oracle(gko, N):
    """Mixed Jacobi-CG on variable-coefficient 3D systems of 4,096-13,824 rows
    (the small-system single-launch inner solves): one restarted
    refinement step to an inner tolerance of 1e-5 takes as many inner
    iterations as the oracle's (within 15%), and the full solve to 1e-10
    needs few refinement steps."""
    G = gko
    A = I.varcoef3d_7pt(N, np.random.default_rng(0))
    b = np.random.default_rng(1).uniform(-1, 1, A.n_rows)
    M = G.from_csr(A)
    _, ro = O.solve_ir(O.CG, A, b, tol=1e-8, max_outer=1, inner_tol=1e-5, inner_maxit=5000, jacobi=True)
    _, rg = solve(G, "cg", M, b, 1e-8, 5000, precision=G.PRECISION_MIXED_F32, refinement=G.REFINE_RESTART,
                  preconditioner=G.PRECOND_JACOBI, max_outer=1, inner_tol=1e-5)
    assert ro.outer_iterations == rg.outer_iterations == 1
    assert abs(rg.iterations - ro.iterations) <= max(3, 0.15 * ro.iterations), (rg, ro)
    assert abs(rg.rel_residual - ro.rel_residual) <= 0.5 * ro.rel_residual
    xg, rg = solve(G, "cg", M, b, 1e-10, 5000, precision=G.PRECISION_MIXED_F32, refinement=G.REFINE_RESTART,
                   preconditioner=G.PRECOND_JACOBI)
    assert rg.status == G.OK and rg.outer_iterations <= 4, rg
    assert np.linalg.norm(b - O.spmv_csr(A, xg)) <= 1.01e-10 * np.linalg.norm(b)
