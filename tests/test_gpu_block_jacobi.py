"""GPU parity of block-Jacobi preconditioning against the CPU oracle, through
the C ABI: the inverse diagonal blocks (bit for bit: both sides run the same
Gauss-Jordan steps with every product and difference rounded on its own),
and block-Jacobi CG / right-preconditioned BiCGSTAB on badly scaled systems
with ragged last blocks."""
import numpy as np
import pytest

import oracle as O
from gpu_util import dev, host
from paper_2006_14290_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def scaled(A, seed=3, spread=3.0):
    """D A D with log-uniform D in [e^-spread, e^spread]."""
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(-spread, spread, A.n_rows))
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    A.val[:] = A.val * s[rows] * s[A.col]
    return A


def csr_from_dense(D, dup=None):
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


def gpu_blocks(G, A, bs):
    B = dev(np.full(A.n_rows * bs, np.nan))
    singular = G.gko_block_jacobi_inverse(G.from_csr(A), bs, B)
    return host(B).reshape(A.n_rows, bs), singular


def random_blocks(n, seed):
    rng = np.random.default_rng(seed)
    D = rng.uniform(-1, 1, (n, n)) * (rng.uniform(0, 1, (n, n)) < 0.4)
    D += np.diag(rng.uniform(0.1, 4, n) * rng.choice([-1, 1], n))
    return csr_from_dense(D, dup=(3, 3, 0.25))


@pytest.mark.parametrize("case,bs", [("random37", 8), ("random37", 5), ("random64", 32), ("varcoef", 1),
                                     ("varcoef", 2), ("varcoef", 3), ("varcoef", 8), ("varcoef", 16),
                                     ("varcoef", 32), ("convdiff", 7), ("convdiff", 32)])
def test_block_inverse_matches_oracle_bitwise(gko, case, bs):
    if case == "random37":
        A = random_blocks(37, 1)
    elif case == "random64":
        A = random_blocks(64, 2)
    elif case == "varcoef":
        A = scaled(I.varcoef3d_7pt(10, np.random.default_rng(0)))  # n = 1,000
    else:
        A = scaled(I.convdiff3d_7pt(21, 3.0))  # n = 9,261: ragged for both sizes
    Bo, so = O.block_jacobi_inv(A, bs)
    Bg, sg = gpu_blocks(gko, A, bs)
    assert sg == so
    np.testing.assert_array_equal(Bg, Bo)


def test_block_inverse_pivoting_and_singular_blocks(gko):
    D = np.zeros((5, 5))
    D[0, 1], D[1, 0], D[1, 1] = 2.0, 3.0, 1.0  # needs a row swap
    D[2, 2], D[2, 3], D[3, 2], D[3, 3] = 1.0, 2.0, 2.0, 4.0  # singular: identity rows
    D[4, 4] = 5.0
    D[0, 4], D[4, 0] = 7.0, -9.0
    A = csr_from_dense(D, dup=(4, 4, 1.5))
    Bo, so = O.block_jacobi_inv(A, 2)
    Bg, sg = gpu_blocks(gko, A, 2)
    assert so == sg == 1
    np.testing.assert_array_equal(Bg, Bo)
    np.testing.assert_array_equal(Bg[2:4], np.eye(2))


def solve(G, name, M, b, tol, maxit, **opt):
    xd = dev(np.zeros(b.size))
    fn = G.gko_solve_cg if name == "cg" else G.gko_solve_bicgstab
    res = fn(M, dev(b), xd, tol, maxit, G.opts(**opt))
    return host(xd), res


def iters_close(a, b):
    return abs(a - b) <= max(2, 0.1 * max(a, b))


@pytest.mark.parametrize("name,bs", [("cg", 1), ("cg", 4), ("cg", 8), ("cg", 32), ("bicgstab", 2),
                                     ("bicgstab", 8), ("bicgstab", 16)])
def test_block_jacobi_solve_matches_oracle(gko, name, bs):
    G = gko
    # n = 1,681 and 1,331: the last block is short for every block size above 1
    A = scaled(I.laplace2d_5pt(41) if name == "cg" else I.convdiff3d_7pt(11, 3.0))
    b = np.random.default_rng(9).uniform(-1, 1, A.n_rows)
    which = O.CG if name == "cg" else O.BICGSTAB
    xo, ro = O.solve_block_jacobi(which, A, b, bs, tol=1e-12, maxit=20000)
    xg, rg = solve(G, name, G.from_csr(A), b, 1e-12, 20000, preconditioner=G.PRECOND_BLOCK_JACOBI,
                   block_size=bs)
    assert ro.status == 0 and rg.status == G.OK, (ro, rg)
    assert rg.rel_residual <= 1e-12
    assert np.linalg.norm(b - O.spmv_csr(A, xg)) <= 1.01e-12 * np.linalg.norm(b)
    assert np.linalg.norm(xg - xo) <= 1e-8 * np.linalg.norm(xo)
    assert iters_close(rg.iterations, ro.iterations), (rg.iterations, ro.iterations)


@pytest.mark.parametrize("name", ["cg", "bicgstab"])
def test_block_jacobi_mid_size_matches_oracle(gko, name):
    """64,000 rows (variable-coefficient 3D Poisson for CG, convection-
    diffusion for BiCGSTAB), default block size 8: iteration counts and
    solutions agree with the oracle, and the default equals block_size=8."""
    G = gko
    A = scaled(I.varcoef3d_7pt(40, np.random.default_rng(1)) if name == "cg" else I.convdiff3d_7pt(40, 2.0),
               spread=2.0)
    b = np.random.default_rng(5).uniform(-1, 1, A.n_rows)
    which = O.CG if name == "cg" else O.BICGSTAB
    xo, ro = O.solve_block_jacobi(which, A, b, 8, tol=1e-10, maxit=20000)
    M = G.from_csr(A)
    xg, rg = solve(G, name, M, b, 1e-10, 20000, preconditioner=G.PRECOND_BLOCK_JACOBI)
    assert ro.status == 0 and rg.status == G.OK, (ro, rg)
    assert np.linalg.norm(b - O.spmv_csr(A, xg)) <= 1.01e-10 * np.linalg.norm(b)
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)
    assert iters_close(rg.iterations, ro.iterations), (rg.iterations, ro.iterations)
    x8, r8 = solve(G, name, M, b, 1e-10, 20000, preconditioner=G.PRECOND_BLOCK_JACOBI, block_size=8)
    assert r8.iterations == rg.iterations
    np.testing.assert_array_equal(x8, xg)


@pytest.mark.parametrize("name", ["cg", "bicgstab"])
def test_block_jacobi_block_diagonal_system_one_step(gko, name):
    """M = A for a block-diagonal A with blocks of bs rows (last one short):
    one preconditioned iteration solves the system."""
    G = gko
    rng = np.random.default_rng(11)
    n, bs = 1003, 8
    D = np.zeros((n, n))
    for base in range(0, n, bs):
        nb = min(bs, n - base)
        Q = rng.uniform(-1, 1, (nb, nb))
        D[base:base + nb, base:base + nb] = Q @ Q.T + nb * np.eye(nb) if name == "cg" else Q + 3 * np.eye(nb)
    A = csr_from_dense(D)
    b = rng.uniform(-1, 1, n)
    xg, rg = solve(G, name, G.from_csr(A), b, 1e-12, 10, preconditioner=G.PRECOND_BLOCK_JACOBI, block_size=bs)
    assert rg.status == G.OK and rg.iterations == 1, rg
    np.testing.assert_allclose(xg, np.linalg.solve(D, b), rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("name,bs,refine", [("cg", 8, "restart"), ("cg", 8, "reliable"), ("cg", 32, "reliable"),
                                            ("bicgstab", 4, "restart"), ("bicgstab", 4, "reliable")])
def test_block_jacobi_mixed_precision_matches_oracle(gko, name, bs, refine):
    """Mixed precision with the FP32-rounded inverse blocks in the FP32
    recurrences: restarted refinement (the library's adaptive inner
    tolerance) and reliable updates against the oracle's same schemes."""
    G = gko
    A = scaled(I.laplace2d_5pt(41) if name == "cg" else I.convdiff3d_7pt(11, 3.0), spread=2.0)
    b = O.spmv_csr(A, np.ones(A.n_rows))
    which = O.CG if name == "cg" else O.BICGSTAB
    M = G.from_csr(A)
    if refine == "restart":
        xo, ro = O.solve_ir(which, A, b, tol=1e-10, inner_tol=1e-5, inner_maxit=5000, adaptive=True,
                            block_size=bs)
        xg, rg = solve(G, name, M, b, 1e-10, 5000, precision=G.PRECISION_MIXED_F32, inner_tol=1e-5,
                       inner_maxit=5000, preconditioner=G.PRECOND_BLOCK_JACOBI, block_size=bs,
                       refinement=G.REFINE_RESTART)
        assert abs(rg.outer_iterations - ro.outer_iterations) <= 1, (rg, ro)
    else:
        xo, ro = O.solve_reliable(which, A, b, tol=1e-12, maxit=5000, delta=0.1, block_size=bs)
        xg, rg = solve(G, name, M, b, 1e-12, 5000, precision=G.PRECISION_MIXED_F32,
                       preconditioner=G.PRECOND_BLOCK_JACOBI, block_size=bs, refinement=G.REFINE_RELIABLE)
        assert abs(rg.iterations - ro.iterations) <= max(3, 0.15 * ro.iterations), (rg, ro)
    tol = 1e-10 if refine == "restart" else 1e-12
    assert ro.status == 0 and rg.status == G.OK, (ro, rg)
    assert rg.rel_residual <= tol
    assert np.linalg.norm(b - O.spmv_csr(A, xg)) <= 1.01 * tol * np.linalg.norm(b)
    assert np.linalg.norm(xg - np.ones(A.n_rows)) <= 1e-6 * np.sqrt(A.n_rows)


def test_block_jacobi_refusals(gko):
    G = gko
    A = I.laplace2d_5pt(8)
    M = G.from_csr(A)
    b = dev(np.ones(A.n_rows))
    bj = G.PRECOND_BLOCK_JACOBI
    cases = [
        (G.gko_solve_gmres, M, G.opts(preconditioner=bj), G.NOT_SUPPORTED),
        (G.gko_solve_cg, M, G.opts(preconditioner=bj, block_size=33), G.INVALID_ARG),
        (G.gko_solve_bicgstab, G.gko_matrix_convert_to_ell(M), G.opts(preconditioner=bj), G.NOT_SUPPORTED),
    ]
    for fn, H, o, want in cases:
        with pytest.raises(G.GkoError) as e:
            fn(H, b, dev(np.zeros(A.n_rows)), 1e-8, 100, o)
        assert e.value.status == want
    for bad in (0, 33):
        with pytest.raises(G.GkoError) as e:
            G.gko_block_jacobi_inverse(M, bad, dev(np.zeros(A.n_rows * 40)))
        assert e.value.status == G.INVALID_ARG
