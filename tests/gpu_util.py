"""Helpers of the GPU parity tests: uploads, the tolerance checks and
oracle-side value rounding.  Expected values always come from ``oracle``."""
import numpy as np

import oracle as O

U64 = 2.0**-53
U32 = 2.0**-24
SPMV_RTOL = 1e-13  # FP64 SpMV: componentwise, relative to sum |alpha a x| + |beta y|


def dev(a, dtype=None):
    import torch

    a = np.ascontiguousarray(a if dtype is None else np.asarray(a, dtype=dtype))
    return torch.from_numpy(a).cuda()


def host(t):
    import torch

    torch.cuda.synchronize()
    return t.cpu().numpy()


def bf16_round(v):
    """Round FP64 values to the nearest bfloat16 (ties to even) on the CPU."""
    v = np.asarray(v, dtype=np.float64)
    m, e = np.frexp(v)
    return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)


def rows_subset(A, idx):
    """CSR of the selected rows (full column space)."""
    from paper_2006_14290_gb300.inputs import Csr

    idx = np.asarray(idx, dtype=np.int64)
    starts = A.row_ptr[idx].astype(np.int64)
    ends = A.row_ptr[idx + 1].astype(np.int64)
    lens = ends - starts
    rp = np.zeros(idx.size + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    take = np.concatenate([np.arange(s, e) for s, e in zip(starts, ends)]) if idx.size else np.zeros(0, np.int64)
    return Csr(idx.size, A.n_cols, rp.astype(np.int32), A.col[take], A.val[take])


def with_values(A, val):
    from paper_2006_14290_gb300.inputs import Csr

    return Csr(A.n_rows, A.n_cols, A.row_ptr, A.col, np.asarray(val, dtype=np.float64), A.name)


def check_spmv_f64(y, A, x, alpha, beta, y0):
    """|y - y_oracle| <= 1e-13 * s_i; rows that miss are re-judged against the
    compensated (near-exact) oracle so that only real errors fail."""
    yo = O.spmv_csr(A, x, alpha, beta, y0)
    s = O.spmv_abs_scale(A, x, alpha, beta, y0)
    nan = np.isnan(yo)
    assert np.array_equal(np.isnan(y), nan), "NaN pattern differs from the oracle"
    err = np.abs(y - yo)
    bad = ~nan & ~(err <= SPMV_RTOL * s)
    if bad.any():
        ye = O.spmv_csr_exact(A, x, alpha, beta, y0)
        bad &= ~(np.abs(y - ye) <= SPMV_RTOL * s)
    assert not bad.any(), f"{int(bad.sum())} rows off, worst {np.max((err / np.maximum(s, 1e-300))[bad]):.3e}"


def check_spmv_f32(y, A, x, alpha, beta, y0, vals32):
    """FP32 values/vectors: both sides within (len+2) u32 s_i of the exact sum."""
    A32 = with_values(A, vals32)
    x32 = np.asarray(x, np.float32)
    y032 = None if y0 is None else np.asarray(y0, np.float32)
    yo = O.spmv_csr_f32(A32, x32, alpha, beta, y032)
    xs = x32.astype(np.float64)
    ys = None if y032 is None else y032.astype(np.float64)
    s = O.spmv_abs_scale(A32, xs, alpha, beta, ys)
    lens = np.diff(A.row_ptr.astype(np.int64))
    nan = np.isnan(yo)
    assert np.array_equal(np.isnan(y), nan), "NaN pattern differs from the oracle"
    err = np.abs(y.astype(np.float64) - yo.astype(np.float64))
    tol = 2 * (lens + 3) * U32 * s + 1e-37
    bad = ~nan & ~(err <= tol)
    assert not bad.any(), f"{int(bad.sum())} rows off"
