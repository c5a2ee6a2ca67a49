"""The bench's algorithmic bytes per SpMV against the arrays they count: each
stored value and index read once (padding excluded), x read once, y written
once.  CPU only."""
import numpy as np

import bench
from paper_2006_14290_gb300 import inputs as I


def arrays_bytes(A, fmt, sv, sx=None, sy=None, ell_width=None):
    sx = sv if sx is None else sx
    sy = sv if sy is None else sy
    L = A.row_lengths()
    xy = sx * A.n_cols + sy * A.n_rows
    if fmt == "csr":  # values, column indices, row pointers
        return A.nnz * sv + A.col.nbytes + A.row_ptr.nbytes + xy
    if fmt == "coo":  # values, column and row index per entry
        rows = np.repeat(np.arange(A.n_rows, dtype=np.int32), L)
        return A.nnz * sv + A.col.nbytes + rows.nbytes + xy
    if fmt == "ell":  # stored (non-padding) entries: value + column index
        return int(L.sum()) * (sv + 4) + xy
    # hybrid: the first min(len, K) entries of a row in ELL, the rest in COO
    ell = np.minimum(L, ell_width)
    tail = L - ell
    return int(ell.sum()) * (sv + 4) + int(tail.sum()) * (sv + 8) + xy


def test_spmv_bytes_match_the_arrays():
    rng = np.random.default_rng(4)
    for A in (I.stencil3d_27pt(6), I.rows_csr([0, 3, 9, 1, 0, 17, 2], 40, rng), I.powerlaw(500, seed=2)):
        L = A.row_lengths()
        for sv in (8, 4, 2):
            for fmt in ("csr", "coo", "ell"):
                got = bench.spmv_bytes(fmt, A.n_rows, A.n_cols, A.nnz, 0, 0, sv, sv, sv)
                assert got == arrays_bytes(A, fmt, sv), (fmt, sv)
            K = 3
            ell_nnz = int(np.minimum(L, K).sum())
            got = bench.spmv_bytes("hybrid", A.n_rows, A.n_cols, A.nnz, ell_nnz, A.nnz - ell_nnz, sv, sv, sv)
            assert got == arrays_bytes(A, "hybrid", sv, ell_width=K)


def test_roofline_case_bytes_closed_form():
    """27-point stencil 128^3 in FP64 COO, the bench's roofline case: n = 128^3,
    nnz = (3*128 - 2)^3, 16 bytes per entry plus x and y."""
    n, nnz = 128 ** 3, (3 * 128 - 2) ** 3
    assert nnz == 55_742_968
    assert bench.spmv_bytes("coo", n, n, nnz, 0, 0, 8, 8, 8) == 925_441_920
    assert I.stencil3d_27pt(10).nnz == (3 * 10 - 2) ** 3
