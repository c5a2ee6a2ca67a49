"""GPU parity of the Krylov solvers (CG, BiCGSTAB, GMRES) and of
mixed-precision iterative refinement against the CPU oracle, through the C ABI.

Readings used here (the paper states no solver algorithm):
* solution parity: both sides solve to 1e-12, then ||x_gpu - x_oracle|| <=
  1e-8 ||x_oracle|| (kappa * 1e-12 << 1e-8 for these systems);
* the reported residual is the true ||b - A x|| / ||b||, recomputed here with
  the oracle's SpMV;
* iteration counts agree within 10% or 2 (GMRES orthogonalises with CGS2 on
  the GPU and MGS in the oracle, which changes rounding only).
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import dev, host
from paper_2006_14290_gb300 import inputs as I

pytestmark = pytest.mark.gpu
SOLVERS = {"cg": O.CG, "bicgstab": O.BICGSTAB, "gmres": O.GMRES}


def gpu_solve(G, name, M, b, x0=None, tol=1e-10, maxit=5000, **opt):
    xd = dev(np.zeros(b.size) if x0 is None else x0)
    fn = {"cg": G.gko_solve_cg, "bicgstab": G.gko_solve_bicgstab, "gmres": G.gko_solve_gmres}[name]
    res = fn(M, dev(b), xd, tol, maxit, G.opts(**opt) if opt else None)
    return host(xd), res


def true_rel_res(A, x, b):
    return float(np.linalg.norm(b - O.spmv_csr(A, x)) / np.linalg.norm(b))


def iters_close(a, b):
    return abs(a - b) <= max(2, 0.1 * max(a, b))


def spd_problem():
    A = I.varcoef3d_7pt(12, np.random.default_rng(5))
    b = np.random.default_rng(6).uniform(-1, 1, A.n_rows)
    return A, b


def nonsym_problem(N=10, P=10.0):
    A = I.convdiff3d_7pt(N, P)
    b = O.spmv_csr(A, np.ones(A.n_rows))
    return A, b


def test_cg_laplace2d_64_matches_oracle(gko):
    G = gko
    A, x, b = I.laplace2d_problem(64)
    M = G.from_csr(A)
    xg, res = gpu_solve(G, "cg", M, b, tol=1e-10)
    xo, ro = O.cg(A, b, tol=1e-10, maxit=5000)
    assert res.status == G.OK and ro.status == 0
    assert res.rel_residual <= 1e-10 and true_rel_res(A, xg, b) <= 1.01e-10
    assert abs(res.rel_residual - true_rel_res(A, xg, b)) <= 1e-13
    assert iters_close(res.iterations, ro.iterations)
    xg12, _ = gpu_solve(G, "cg", M, b, tol=1e-12)
    xo12, _ = O.cg(A, b, tol=1e-12, maxit=5000)
    assert np.linalg.norm(xg12 - xo12) <= 1e-8 * np.linalg.norm(xo12)


@pytest.mark.parametrize("fmt", ["csr", "ell", "coo", "hybrid", "sellp"])
@pytest.mark.parametrize("name", ["cg", "bicgstab", "gmres"])
def test_solvers_all_formats(gko, fmt, name):
    G = gko
    A, b = spd_problem() if name == "cg" else nonsym_problem()
    M = G.from_csr(A)
    if fmt == "ell":
        M = G.gko_matrix_convert_to_ell(M)
    elif fmt == "coo":
        M = G.gko_matrix_convert_to_coo(M)
    elif fmt == "hybrid":
        M = G.gko_matrix_convert_to_hybrid(M, 3)
    elif fmt == "sellp":
        M = G.gko_matrix_convert_to_sellp(M, 32)
    xg, res = gpu_solve(G, name, M, b, tol=1e-12, maxit=4000)
    xo, ro = O.solve(SOLVERS[name], A, b, tol=1e-12, maxit=4000)
    assert res.status == G.OK and ro.status == 0, (res, ro)
    assert res.rel_residual <= 1e-12
    assert true_rel_res(A, xg, b) <= 1.01e-12
    assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)
    if name != "gmres":
        assert iters_close(res.iterations, ro.iterations), (res.iterations, ro.iterations)
    else:
        assert iters_close(res.iterations, ro.iterations) or abs(res.outer_iterations - ro.outer_iterations) <= 1


@pytest.mark.parametrize("plan", [(0, 4, 2), (2, 1, 1), (3, 1, 1)], ids=["subwarp", "merge", "nzsplit"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("name", ["cg", "bicgstab", "gmres"])
def test_solvers_every_csr_plan(gko, plan, precision, name):
    """The solvers on CSR plans whose SpMV does not fuse the dot product
    (subwarp, merge path, nonzero split); mixed precision runs the plan on the
    solver's cached FP32 copy."""
    G = gko
    A, b = spd_problem() if name == "cg" else nonsym_problem()
    M = G.from_csr(A)
    M.set_plan(*plan, 1024)
    assert M.plan()["kernel"] == plan[0]
    opt = {} if precision == "f64" else {"precision": G.PRECISION_MIXED_F32}
    xg, res = gpu_solve(G, name, M, b, tol=1e-12, maxit=4000, **opt)
    xo, ro = O.solve(SOLVERS[name], A, b, tol=1e-12, maxit=4000)
    assert res.status == G.OK and ro.status == 0, (res, ro)
    assert true_rel_res(A, xg, b) <= 1.01e-12
    assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)
    if precision == "f64" and name != "gmres":
        assert iters_close(res.iterations, ro.iterations), (res.iterations, ro.iterations)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("name", ["cg", "bicgstab", "gmres"])
def test_solvers_mid_size_match_oracle(gko, name, precision):
    """Solution parity on a grid-sized launch (n = 48^3 = 110,592: many full
    waves of every vector kernel and of the SpMV): 7-point Poisson (CG, b
    uniform in [-1, 1]) and upwind convection-diffusion at cell Peclet 1
    (BiCGSTAB, GMRES(30), b = A*1), both sides to 1e-12, FP64 and mixed FP32."""
    G = gko
    if name == "cg":
        A = I.stencil3d_7pt(48)
        b = np.random.default_rng(11).uniform(-1, 1, A.n_rows)
    else:
        A = I.convdiff3d_7pt(48, 1.0)
        b = O.spmv_csr(A, np.ones(A.n_rows))
    M = G.from_csr(A)
    opt = {} if precision == "f64" else {"precision": G.PRECISION_MIXED_F32}
    xg, res = gpu_solve(G, name, M, b, tol=1e-12, maxit=6000, **opt)
    xo, ro = O.solve(SOLVERS[name], A, b, tol=1e-12, maxit=6000)
    assert res.status == G.OK and ro.status == 0, (res, ro)
    assert true_rel_res(A, xg, b) <= 1.01e-12
    assert abs(res.rel_residual - true_rel_res(A, xg, b)) <= 1e-13
    assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)
    if precision == "f64" and name != "gmres":
        assert iters_close(res.iterations, ro.iterations), (res.iterations, ro.iterations)


@pytest.mark.parametrize("restart", [5, 30])
def test_gmres_restart_lengths(gko, restart):
    G = gko
    A, b = nonsym_problem(12, 3.0)
    M = G.from_csr(A)
    xg, res = gpu_solve(G, "gmres", M, b, tol=1e-11, maxit=5000, restart=restart)
    xo, ro = O.gmres(A, b, tol=1e-11, maxit=5000, restart=restart)
    assert res.status == G.OK and res.rel_residual <= 1e-11
    assert iters_close(res.iterations, ro.iterations), (res, ro)
    assert np.max(np.abs(xg - 1.0)) < 1e-7


@pytest.mark.parametrize("precision", ["f32", "bf16"])
@pytest.mark.parametrize("name", ["cg", "bicgstab", "gmres"])
def test_mixed_precision_refinement(gko, precision, name):
    G = gko
    A, b = spd_problem() if name == "cg" else nonsym_problem()
    M = G.from_csr(A)
    prec = G.PRECISION_MIXED_F32 if precision == "f32" else G.PRECISION_MIXED_BF16
    xg, res = gpu_solve(G, name, M, b, tol=1e-12, maxit=2000, precision=prec,
                        inner_tol=1e-3 if precision == "bf16" else 1e-4, refinement=G.REFINE_RESTART)
    assert res.status == G.OK, res
    assert res.outer_iterations >= 2
    assert res.rel_residual <= 1e-12 and true_rel_res(A, xg, b) <= 1.01e-12
    xo, _ = O.solve(SOLVERS[name], A, b, tol=1e-12, maxit=4000)
    assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)
    if precision == "f32":
        # the library's default inner limits: GMRES 4 restart cycles per
        # refinement step (outer steps up to max(30, ceil(maxit / 120))), the
        # others the whole iteration budget
        inner = dict(inner_maxit=120, max_outer=30) if name == "gmres" else dict(inner_maxit=2000)
        xi, ri = O.solve_ir(SOLVERS[name], A, b, tol=1e-12, inner_tol=1e-4, adaptive=True, **inner)
        assert ri.status == 0 and abs(res.outer_iterations - ri.outer_iterations) <= 2, (res, ri)


@pytest.mark.parametrize("fmt", ["csr", "ell", "coo"])
@pytest.mark.parametrize("precision", ["f32", "bf16"])
@pytest.mark.parametrize("name", ["cg", "bicgstab"])
def test_reliable_updates_match_oracle(gko, name, precision, fmt):
    """Mixed precision with reliable updates: FP32 (or BF16-valued) recurrences
    with FP32 vectors, the partial solution folded into the FP64 x and the
    residual replaced by the FP64 one; both sides to 1e-12, solution parity
    with the oracle's reliable-update solve (FP32 values; BF16 rounds A
    further, so there only the residual and the FP64 solution are judged);
    update counts are of the same order (the GPU applies FP64 scalars to FP32
    vectors as float pairs, the oracle in FP64 then rounds)."""
    G = gko
    A, b = spd_problem() if name == "cg" else nonsym_problem(10, 3.0)
    M = G.from_csr(A)
    if fmt == "ell":
        M = G.gko_matrix_convert_to_ell(M)
    elif fmt == "coo":
        M = G.gko_matrix_convert_to_coo(M)
    prec = G.PRECISION_MIXED_F32 if precision == "f32" else G.PRECISION_MIXED_BF16
    xg, res = gpu_solve(G, name, M, b, tol=1e-12, maxit=5000, precision=prec, refinement=G.REFINE_RELIABLE)
    assert res.status == G.OK, res
    assert res.rel_residual <= 1e-12 and true_rel_res(A, xg, b) <= 1.01e-12
    assert abs(res.rel_residual - true_rel_res(A, xg, b)) <= 1e-13
    xo, ro = O.solve(SOLVERS[name], A, b, tol=1e-12, maxit=5000)
    assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)
    if precision == "f32":
        xr, rr = O.solve_reliable(SOLVERS[name], A, b, tol=1e-12, maxit=5000, delta=0.1)
        assert rr.status == 0 and np.linalg.norm(xg - xr) <= 1e-8 * np.linalg.norm(xr)
        assert abs(res.iterations - rr.iterations) <= max(3, 0.15 * rr.iterations), (res, rr)
        assert abs(res.outer_iterations - rr.outer_iterations) <= max(2, 0.3 * rr.outer_iterations), (res, rr)


@pytest.mark.parametrize("name", ["cg", "bicgstab"])
def test_reliable_updates_large_default(gko, name):
    """The library's default mixed-precision path above 2^18 rows: reliable
    updates with the FP32 copy stored in ELL (rows of near-equal length),
    against the oracle's reliable-update solve (FP32 CSR recurrences; the ELL
    copy sums each row in the same storage order) and its FP64 solve, both
    sides to 1e-12: n = 65^3 = 274,625."""
    G = gko
    if name == "cg":
        A = I.stencil3d_7pt(65)
        b = np.random.default_rng(12).uniform(-1, 1, A.n_rows)
    else:
        A = I.convdiff3d_7pt(65, 1.0)
        b = O.spmv_csr(A, np.ones(A.n_rows))
    assert A.n_rows > 1 << 18
    M = G.from_csr(A)
    G.gko_matrix_convert_to_ell(M, 1.2)  # the copy's format rule accepts this matrix
    xg, res = gpu_solve(G, name, M, b, tol=1e-12, maxit=5000, precision=G.PRECISION_MIXED_F32)
    assert res.status == G.OK and res.outer_iterations >= 3, res
    assert true_rel_res(A, xg, b) <= 1.01e-12
    assert abs(res.rel_residual - true_rel_res(A, xg, b)) <= 1e-13
    xr, rr = O.solve_reliable(SOLVERS[name], A, b, tol=1e-12, maxit=5000, delta=0.1)
    assert rr.status == 0 and np.linalg.norm(xg - xr) <= 1e-8 * np.linalg.norm(xr)
    assert abs(res.iterations - rr.iterations) <= max(3, 0.15 * rr.iterations), (res, rr)
    xo, ro = O.solve(SOLVERS[name], A, b, tol=1e-12, maxit=5000)
    assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)


def test_reliable_updates_options(gko):
    """Refinement options: GMRES refuses reliable updates, bad modes and
    factors are refused, delta = 0 updates only at convergence, x0 and b = 0
    behave as in the other solves, and the iteration cap holds."""
    G = gko
    A, b = nonsym_problem(8, 3.0)
    M = G.from_csr(A)
    mixed = dict(precision=G.PRECISION_MIXED_F32)
    for bad in (dict(refinement=7), dict(refinement=G.REFINE_RELIABLE, reliable_delta=1.5),
                dict(refinement=G.REFINE_RELIABLE, reliable_delta=-0.1)):
        with pytest.raises(G.GkoError) as e:
            gpu_solve(G, "bicgstab", M, b, **mixed, **bad)
        assert e.value.status == G.INVALID_ARG
    with pytest.raises(G.GkoError) as e:
        gpu_solve(G, "gmres", M, b, **mixed, refinement=G.REFINE_RELIABLE)
    assert e.value.status == G.NOT_SUPPORTED
    for name in ("cg", "bicgstab"):
        A2, b2 = spd_problem() if name == "cg" else (A, b)
        M2 = G.from_csr(A2)
        x, res = gpu_solve(G, name, M2, np.zeros(A2.n_rows), x0=np.ones(A2.n_rows), **mixed,
                           refinement=G.REFINE_RELIABLE)
        assert res.status == G.OK and res.iterations == 0 and np.all(x == 0)
        xs, _ = O.solve(SOLVERS[name], A2, b2, tol=1e-14, maxit=5000)
        x, res = gpu_solve(G, name, M2, b2, x0=xs, tol=1e-10, **mixed, refinement=G.REFINE_RELIABLE)
        assert res.status == G.OK and res.iterations == 0
        x, res = gpu_solve(G, name, M2, b2, tol=1e-14, maxit=3, **mixed, refinement=G.REFINE_RELIABLE)
        assert res.status == G.NOT_CONVERGED and res.iterations == 3
        assert abs(res.rel_residual - true_rel_res(A2, x, b2)) <= 1e-12
        x0 = np.random.default_rng(1).uniform(-1, 1, A2.n_rows)
        x, res = gpu_solve(G, name, M2, b2, x0=x0, tol=1e-10, maxit=5000, **mixed, refinement=G.REFINE_RELIABLE,
                           reliable_delta=0.01)
        assert res.status == G.OK and true_rel_res(A2, x, b2) <= 1.01e-10
        x2, res2 = gpu_solve(G, name, M2, b2, x0=x0, tol=1e-10, maxit=5000, **mixed,
                             refinement=G.REFINE_RELIABLE, reliable_delta=0.01)
        assert x.tobytes() == x2.tobytes() and res.iterations == res2.iterations


@pytest.mark.parametrize("N", [128, 129])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_cg_small_system_paths_match_oracle(gko, N, precision):
    """CG on 2D systems at the edge of the one-cluster CG (n = 128^2 = 16,384,
    16 CTAs of 256 threads x 4 rows) and just past it (n = 129^2, the
    cooperative-grid CG): solution parity with the oracle at 1e-12, FP64 and
    mixed FP32 (restarted refinement, whose FP32 inner solves take the
    cooperative-grid kernel), with and without Jacobi."""
    G = gko
    A = I.varcoef2d_5pt(N, np.random.default_rng(N))
    b = np.random.default_rng(3).uniform(-1, 1, A.n_rows)
    M = G.from_csr(A)
    opt = {} if precision == "f64" else {"precision": G.PRECISION_MIXED_F32, "refinement": G.REFINE_RESTART}
    xo, ro = O.cg(A, b, tol=1e-12, maxit=20000)
    for pc in (G.PRECOND_NONE, G.PRECOND_JACOBI):
        xg, res = gpu_solve(G, "cg", M, b, tol=1e-12, maxit=20000, preconditioner=pc, **opt)
        assert res.status == G.OK, res
        assert true_rel_res(A, xg, b) <= 1.01e-12
        assert abs(res.rel_residual - true_rel_res(A, xg, b)) <= 1e-13
        assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)
        if precision == "f64" and pc == G.PRECOND_NONE:
            assert iters_close(res.iterations, ro.iterations), (res.iterations, ro.iterations)


def test_edge_cases(gko):
    G = gko
    A, b = spd_problem()
    M = G.from_csr(A)
    for name in ("cg", "bicgstab", "gmres"):
        x, res = gpu_solve(G, name, M, np.zeros(A.n_rows), x0=np.ones(A.n_rows))
        assert res.status == G.OK and res.iterations == 0 and np.all(x == 0)
        xs, _ = O.cg(A, b, tol=1e-14, maxit=5000)
        x, res = gpu_solve(G, name, M, b, x0=xs, tol=1e-10)
        assert res.status == G.OK and res.iterations == 0
        x, res = gpu_solve(G, name, M, b, maxit=0)
        assert res.status == G.NOT_CONVERGED and res.iterations == 0
        x, res = gpu_solve(G, name, M, b, tol=1e-14, maxit=3)
        assert res.status == G.NOT_CONVERGED and res.iterations == 3 and res.rel_residual > 1e-6
        assert abs(res.rel_residual - true_rel_res(A, x, b)) <= 1e-12
    D = I.Csr(2, 2, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, -1.0]))
    x, res = gpu_solve(G, "cg", G.from_csr(D), np.array([1.0, 1.0]))
    assert res.status == G.BREAKDOWN


@pytest.mark.parametrize("name", ["cg", "bicgstab", "gmres"])
def test_nonzero_x0_and_determinism(gko, name):
    G = gko
    A, b = spd_problem() if name == "cg" else nonsym_problem()
    M = G.from_csr(A)
    x0 = np.random.default_rng(1).uniform(-1, 1, A.n_rows)
    x1, r1 = gpu_solve(G, name, M, b, x0=x0, tol=1e-11)
    x2, r2 = gpu_solve(G, name, M, b, x0=x0, tol=1e-11)
    assert r1.status == G.OK and x1.tobytes() == x2.tobytes() and r1.iterations == r2.iterations
    xo, ro = O.solve(SOLVERS[name], A, b, x0=x0, tol=1e-11, maxit=5000)
    assert iters_close(r1.iterations, ro.iterations) or name == "gmres"
    assert true_rel_res(A, x1, b) <= 1.01e-11


@pytest.mark.slow
def test_cg_poisson_256_full_size(gko):
    """The CG workload of the solver benchmark (7-point 256^3, b = A*1), FP64
    and mixed FP32, checked with the oracle's SpMV."""
    import torch

    G = gko
    A = I.stencil3d_7pt(256)
    M = G.from_csr(A)
    ones = torch.ones(A.n_rows, dtype=torch.float64, device="cuda")
    bd = torch.zeros_like(ones)
    G.gko_spmv(1.0, M, ones, 0.0, bd)
    b = host(bd)
    for prec in (G.PRECISION_F64, G.PRECISION_MIXED_F32):
        xd = torch.zeros_like(ones)
        res = G.gko_solve_cg(M, bd, xd, 1e-8, 5000, G.opts(precision=prec))
        assert res.status == G.OK, res
        x = host(xd)
        assert true_rel_res(A, x, b) <= 1.01e-8
        assert abs(res.rel_residual - true_rel_res(A, x, b)) <= 1e-11


@pytest.mark.slow
@pytest.mark.parametrize("case", ["bicgstab_P1", "gmres30_P10", "cg_jacobi_varcoef"])
def test_solver_workloads_full_size(gko, case):
    """The other solver workloads of the benchmark at full size (128^3), FP64
    and mixed FP32, in the benchmark's options: converged, the reported
    residual equals the true one recomputed with the oracle's SpMV, and the
    iterate is close to the exact solution 1 (b = A*1)."""
    import torch

    G = gko
    if case == "cg_jacobi_varcoef":
        A = I.varcoef3d_7pt(128, np.random.default_rng(0))
    else:
        A = I.convdiff3d_7pt(128, 1.0 if case == "bicgstab_P1" else 10.0)
    M = G.from_csr(A)
    ones = torch.ones(A.n_rows, dtype=torch.float64, device="cuda")
    bd = torch.zeros_like(ones)
    G.gko_spmv(1.0, M, ones, 0.0, bd)
    b = host(bd)
    fn = {"bicgstab_P1": G.gko_solve_bicgstab, "gmres30_P10": G.gko_solve_gmres,
          "cg_jacobi_varcoef": G.gko_solve_cg}[case]
    pc = G.PRECOND_JACOBI if case == "cg_jacobi_varcoef" else G.PRECOND_NONE
    for prec in (G.PRECISION_F64, G.PRECISION_MIXED_F32):
        xd = torch.zeros_like(ones)
        res = fn(M, bd, xd, 1e-8, 20000, G.opts(precision=prec, restart=30, inner_maxit=2000, max_outer=12,
                                                 preconditioner=pc))
        assert res.status == G.OK, (case, prec, res)
        x = host(xd)
        tr = true_rel_res(A, x, b)
        assert tr <= 1.01e-8 and abs(res.rel_residual - tr) <= 1e-11
        assert np.linalg.norm(x - 1.0) <= 1e-4 * np.sqrt(A.n_rows)
