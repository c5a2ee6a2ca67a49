"""The allocation-free COO SpMV (gko_spmv_coo_noalloc) against gko_spmv.

gko_spmv_coo_noalloc serves callers that cannot allocate device memory when
they multiply; it keeps its tile carries in a fixed device array inside the
library.  Its results must match the pool-scratch path within the SpMV
tolerance on two calls in a row (the array keeps the previous call's
contents), and handles beyond its size limit must be refused.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import check_spmv_f64, dev, host
from paper_2006_14290_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _coo(G, A):
    return G.gko_matrix_convert_to_coo(G.from_csr(A))


@pytest.mark.parametrize("name", ["powerlaw", "stencil", "empty_rows", "stencil_rowblock_plan"])
def test_noalloc_matches_spmv_twice(gko, name):
    G = gko
    rng = np.random.default_rng(3)
    if name == "powerlaw":
        A = I.powerlaw(60000, seed=2)  # long rows spanning several tiles
    elif name.startswith("stencil"):
        A = I.stencil3d_27pt(24)
    else:
        A = I.random_csr(5000, 4000, 0.003, rng, empty_rows=0.4, sort_cols=False)
    M = _coo(G, A)
    if name == "stencil_rowblock_plan":
        # gko_spmv then runs the row-block COO kernel (another summation
        # order); the allocation-free call keeps the segmented reduction
        M.set_plan(1, 4, 1, 1024)
        assert M.plan()["kernel"] == 1
    for call, (alpha, beta) in enumerate([(1.0, 0.0), (-0.5, 2.0)]):
        x = rng.uniform(-1, 1, A.n_cols)
        y0 = rng.uniform(-1, 1, A.n_rows)
        y_ref = dev(y0)
        G.gko_spmv(alpha, M, dev(x), beta, y_ref)
        y_new = dev(y0)
        G.gko_spmv_coo_noalloc(alpha, M, dev(x), beta, y_new)
        r, n = host(y_ref), host(y_new)
        s = O.spmv_abs_scale(A, x, alpha, beta, y0)
        assert np.all(np.abs(n - r) <= 1e-13 * s), f"call {call}"
        check_spmv_f64(n, A, x, alpha, beta, y0)
    G.gko_device_status()


def test_noalloc_refuses_oversized_and_wrong_handles(gko):
    import torch

    G = gko
    with pytest.raises(G.GkoError) as e:
        G.gko_spmv_coo_noalloc(1.0, G.from_csr(I.laplace2d_5pt(8)), dev(np.ones(64)), 0.0, dev(np.zeros(64)))
    assert e.value.status == G.INVALID_ARG
    nnz = (1 << 27) + 1
    rp = torch.arange(nnz + 1, dtype=torch.int32, device="cuda")
    col = torch.zeros(nnz, dtype=torch.int32, device="cuda")
    val = torch.ones(nnz, dtype=torch.float64, device="cuda")
    big = G.gko_matrix_convert_to_coo(G.gko_matrix_create_csr(nnz, 1, rp, col, val))
    del rp, col, val
    with pytest.raises(G.GkoError) as e:
        G.gko_spmv_coo_noalloc(1.0, big, torch.ones(1, dtype=torch.float64, device="cuda"), 0.0,
                               torch.zeros(nnz, dtype=torch.float64, device="cuda"))
    assert e.value.status == G.INVALID_ARG and "at most" in str(e.value)
