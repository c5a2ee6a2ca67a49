"""GPU parity of the BLAS-1 kernels (dot, nrm2, axpy, multi-dot, fused
multi-axpy + norm, fused SpMV + dot) against the oracle, through the C ABI."""
import numpy as np
import pytest

import oracle as O
from gpu_util import U64, dev, host
from paper_2006_14290_gb300 import inputs as I

pytestmark = pytest.mark.gpu
RTOL = 1e-13  # relative to sum |x_i y_i| (reordered FP64 sums)


@pytest.mark.parametrize("n", [0, 1, 1000, 4097, 1_000_003])
def test_dot_nrm2_axpy(gko, n):
    G = gko
    rng = np.random.default_rng(n)
    x = rng.uniform(-1, 1, n)
    y = rng.uniform(-1, 1, n)
    scale = float(np.sum(np.abs(x * y))) if n else 0.0
    d = G.gko_dot(dev(x), dev(y))
    assert abs(d - O.dot(x, y)) <= RTOL * scale + 1e-300
    nr = G.gko_nrm2(dev(x))
    assert abs(nr - np.sqrt(O.dot(x, x))) <= RTOL * (np.sqrt(O.dot(x, x)) + 1e-300)
    yd = dev(y)
    G.gko_axpy(-2.5, dev(x), yd)
    np.testing.assert_allclose(host(yd), O.axpy(-2.5, x, y), rtol=0, atol=4 * U64 * (2.5 + 1))


@pytest.mark.parametrize("n,k", [(10, 1), (5000, 7), (300001, 31)])
def test_multi_dot_and_multi_axpy_norm(gko, n, k):
    G = gko
    rng = np.random.default_rng(k)
    V = rng.uniform(-1, 1, (k, n))
    w = rng.uniform(-1, 1, n)
    h = G.gko_multi_dot(dev(V), dev(w), k)
    ho = O.multi_dot(V, w)
    scale = np.abs(V) @ np.abs(w)
    assert np.all(np.abs(h - ho) <= RTOL * scale)
    y = rng.uniform(-1, 1, n)
    hh = rng.uniform(-0.1, 0.1, k)
    yd = dev(y)
    nr = G.gko_multi_axpy_norm(dev(V), hh, yd)
    yo, nro = O.multi_axpy_norm(V, hh, y)
    tol = (k + 2) * U64 * (np.abs(y) + np.abs(hh) @ np.abs(V))
    assert np.all(np.abs(host(yd) - yo) <= tol)
    assert abs(nr - nro) <= 1e-13 * nro


@pytest.mark.parametrize("fmt", ["csr", "ell", "coo", "hybrid", "sellp"])
def test_spmv_dot(gko, fmt):
    G = gko
    A = I.stencil3d_7pt(20) if fmt != "csr" else I.powerlaw(40000, seed=4)
    M = G.from_csr(A)
    if fmt == "ell":
        M = G.gko_matrix_convert_to_ell(M)
    elif fmt == "coo":
        M = G.gko_matrix_convert_to_coo(M)
    elif fmt == "hybrid":
        M = G.gko_matrix_convert_to_hybrid(M)
    elif fmt == "sellp":
        M = G.gko_matrix_convert_to_sellp(M)
    x = np.random.default_rng(3).uniform(-1, 1, A.n_cols)
    yd = dev(np.zeros(A.n_rows))
    d = G.gko_spmv_dot(M, dev(x), yd)
    y = host(yd)
    yo = O.spmv_csr(A, x)
    s = O.spmv_abs_scale(A, x)
    assert np.all(np.abs(y - yo) <= 1e-13 * s)
    do = O.dot(x, yo)
    assert abs(d - do) <= 1e-12 * float(np.abs(x) @ s)
