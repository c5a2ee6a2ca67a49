"""Thin Python binding of the C ABI in ``include/gko.h``.

Argument marshalling only: every step of the computation runs in the CUDA
library ``libgko_gb300.so``.  Functions keep the C names.  Device vectors
are ``torch`` CUDA tensors (PyTorch provides device memory and streams);
host arrays are numpy arrays.  A non-OK status raises :class:`GkoError`.
There is no CPU fallback: without the built library or a GPU, :func:`load`
raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgko_gb300.so")

OK, INVALID_ARG, OUT_OF_MEMORY, FORMAT_UNSUITABLE, NOT_CONVERGED, BREAKDOWN, TIMEOUT, CUDA_ERROR, \
    BUDGET_EXCEEDED, NOT_SUPPORTED = range(10)
F64, F32, BF16 = 0, 1, 2
CSR, ELL, COO, HYBRID, SELLP = 0, 1, 2, 3, 4
PRECISION_F64, PRECISION_MIXED_F32, PRECISION_MIXED_BF16 = 0, 1, 2
REFINE_AUTO, REFINE_RESTART, REFINE_RELIABLE = 0, 1, 2

_lib = None
_P = C.c_void_p
_I32 = C.c_int32
_I64 = C.c_int64
_D = C.c_double
_PI64 = C.POINTER(C.c_int64)
_PI32 = C.POINTER(C.c_int32)


class GkoError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


class SolveOpts(C.Structure):
    _fields_ = [("restart", C.c_int32), ("precision", C.c_int32), ("inner_tol", C.c_double),
                ("max_outer", C.c_int32), ("inner_maxit", C.c_int32), ("check_every", C.c_int32),
                ("preconditioner", C.c_int32), ("refinement", C.c_int32), ("block_size", C.c_int32),
                ("reliable_delta", C.c_double)]


class SolveResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("outer_iterations", C.c_int32),
                ("reserved", C.c_int32), ("rel_residual", C.c_double)]

    def __repr__(self):
        return (f"SolveResult(status={self.status}, iterations={self.iterations}, "
                f"outer_iterations={self.outer_iterations}, rel_residual={self.rel_residual:.3e})")


# name -> (restype, argtypes); every symbol the header declares
SIGNATURES = {
    "gko_last_error": (C.c_char_p, []),
    "gko_status_string": (C.c_char_p, [C.c_int]),
    "gko_version": (C.c_int, []),
    "gko_device_status": (C.c_int, [_P]),
    "gko_set_memory_budget": (C.c_int, [_I64]),
    "gko_memory_in_use": (C.c_int, [_PI64]),
    "gko_matrix_create_csr": (C.c_int, [_I64, _I64, _I64, _P, _P, _P, C.c_int, C.c_int, _P, C.POINTER(_P)]),
    "gko_matrix_convert_to_ell": (C.c_int, [_P, _D, _P, C.POINTER(_P)]),
    "gko_matrix_convert_to_coo": (C.c_int, [_P, _P, C.POINTER(_P)]),
    "gko_matrix_convert_to_hybrid": (C.c_int, [_P, _I32, _P, C.POINTER(_P)]),
    "gko_matrix_convert_to_sellp": (C.c_int, [_P, _I32, _D, _P, C.POINTER(_P)]),
    "gko_matrix_convert_values": (C.c_int, [_P, C.c_int, _P, C.POINTER(_P)]),
    "gko_matrix_info": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), _PI64, _PI64, _PI64, _PI32,
                                  _PI64, _PI64, _PI64]),
    "gko_matrix_export": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "gko_matrix_plan": (C.c_int, [_P, _PI32, _PI32, _PI32, _PI32, _PI32, _PI64, _PI64, _PI64]),
    "gko_matrix_set_plan": (C.c_int, [_P, _I32, _I32, _I32, _I32, _P]),
    "gko_matrix_tune": (C.c_int, [_P, _P, _P, _I32, _I32, _PI32, _PI32, _PI32, _PI32, C.POINTER(C.c_float),
                                  _P]),
    "gko_matrix_destroy": (C.c_int, [_P]),
    "gko_spmv": (C.c_int, [C.POINTER(_D), _P, _P, C.POINTER(_D), _P, C.c_int, _P]),
    "gko_spmv_coo_noalloc": (C.c_int, [C.POINTER(_D), _P, _P, C.POINTER(_D), _P, _P]),
    "gko_spmv_host": (C.c_int, [C.POINTER(_D), _P, _P, C.POINTER(_D), _P, C.c_int, _P, _P, _P]),
    "gko_bench_subwarp_reduce": (C.c_int, [_I32, _I32, C.c_int, _I32, _P, C.c_int64, _P]),
    "gko_bench_fma": (C.c_int, [C.c_int, _I32, _P, C.c_int64, _P]),
    "gko_bench_gather": (C.c_int, [C.c_int, _I32, _P, _I32, _P, C.c_int64, _P]),
    "gko_diag_bounded_wait": (C.c_int, [C.c_int64, C.POINTER(C.c_int32), _P]),
    "gko_dot": (C.c_int, [_I64, _P, _P, C.POINTER(_D), _P]),
    "gko_nrm2": (C.c_int, [_I64, _P, C.POINTER(_D), _P]),
    "gko_axpy": (C.c_int, [_I64, _D, _P, _P, _P]),
    "gko_multi_axpy_norm": (C.c_int, [_I64, _I32, _P, _P, _I64, _P, C.POINTER(_D), _P]),
    "gko_multi_dot": (C.c_int, [_I64, _I32, _P, _I64, _P, _P, _P]),
    "gko_spmv_dot": (C.c_int, [_P, _P, _P, C.POINTER(_D), _P]),
    "gko_solve_cg": (C.c_int, [_P, _P, _P, _D, _I32, C.POINTER(SolveOpts), C.POINTER(SolveResult), _P]),
    "gko_solve_bicgstab": (C.c_int, [_P, _P, _P, _D, _I32, C.POINTER(SolveOpts), C.POINTER(SolveResult), _P]),
    "gko_solve_gmres": (C.c_int, [_P, _P, _P, _D, _I32, C.POINTER(SolveOpts), C.POINTER(SolveResult), _P]),
    "gko_block_jacobi_inverse": (C.c_int, [_P, _I32, _P, _PI64, _P]),
}
SIGNATURES.update({
    "gko_batch_create": (C.c_int, [_I32, _P, _P, _P, _P, _P, C.c_int, _P, C.POINTER(_P)]),
    "gko_batch_create_systems": (C.c_int, [_I32, _P, _P, _P, _P, C.c_int, _P, C.POINTER(_P)]),
    "gko_batch_export": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "gko_batch_cg": (C.c_int, [_P, _P, _P, _D, _I32, _P, _P, _P, _P]),
    "gko_batch_tune": (C.c_int, [_P, _P, _P, _D, _I32, _PI32, _PI32, _PI32, C.POINTER(C.c_float), _P]),
    "gko_batch_set_threshold": (C.c_int, [_P, _I32, _P]),
    "gko_batch_set_schedule": (C.c_int, [_P, _I32, _I32, _I32, _P]),
    "gko_batch_set_precision": (C.c_int, [_P, _I32, C.c_double, _P]),
    "gko_batch_last_updates": (C.c_int, [_P, _P, _P]),
    "gko_batch_info": (C.c_int, [_P, _PI32, _PI64, _PI64, _PI32, _PI32, _PI32, _PI32]),
    "gko_batch_destroy": (C.c_int, [_P]),
})
SIGNATURES.update({
    "gko_server_create": (C.c_int, [_I32, _I64, C.POINTER(_P)]),
    "gko_server_add_matrix": (C.c_int, [_P, _P, _PI32]),
    "gko_server_submit": (C.c_int, [_P, _I32, _I32, _P, _D, _I32, C.POINTER(SolveOpts), _PI64]),
    "gko_server_result": (C.c_int, [_P, _I64, C.c_int, _PI32, C.POINTER(SolveResult), _P, C.POINTER(_D)]),
    "gko_server_stats": (C.c_int, [_P, _PI64, C.POINTER(_D), C.POINTER(_D), C.POINTER(_D), _PI32]),
    "gko_server_destroy": (C.c_int, [_P]),
})
OPTIONAL = {}


def load(path: str = LIB_PATH):
    """Load the CUDA library (no fallback: raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = C.CDLL(path)
    for name, (ret, args) in {**SIGNATURES, **OPTIONAL}.items():
        f = getattr(L, name, None)
        if f is None:
            if name in SIGNATURES:
                raise RuntimeError(f"{path} does not export {name}")
            continue
        f.restype = ret
        f.argtypes = args
    _lib = L
    return L


def lib():
    return _lib if _lib is not None else load()


def _check(status: int, where: str):
    if status != OK:
        msg = lib().gko_last_error().decode(errors="replace")
        raise GkoError(status, where, msg or lib().gko_status_string(status).decode())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dptr(t):
    """Device pointer of a torch tensor (contiguous)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _hptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


_NP_DTYPE = {F64: np.float64, F32: np.float32}


# ------------------------------------------------------------------ matrices

class Matrix:
    """Owning wrapper of a gko_matrix handle."""

    def __init__(self, handle: C.c_void_p):
        self.handle = handle

    def __del__(self):
        try:
            if self.handle and _lib is not None:
                _lib.gko_matrix_destroy(self.handle)
        except Exception:
            pass
        self.handle = None

    @property
    def _as_param_(self):
        return self.handle

    def info(self):
        fmt, dt = C.c_int(), C.c_int()
        n, m, nnz, stride, coo, nbytes = (C.c_int64() for _ in range(6))
        K = C.c_int32()
        _check(lib().gko_matrix_info(self.handle, C.byref(fmt), C.byref(dt), C.byref(n), C.byref(m), C.byref(nnz),
                                     C.byref(K), C.byref(stride), C.byref(coo), C.byref(nbytes)), "info")
        return dict(format=fmt.value, dtype=dt.value, n_rows=n.value, n_cols=m.value, nnz=nnz.value,
                    ell_width=K.value, ell_stride=stride.value, coo_nnz=coo.value, bytes=nbytes.value)

    def plan(self):
        K, S, R, cap, thr = (C.c_int32() for _ in range(5))
        nl, nc = C.c_int64(), C.c_int64()
        hist = (C.c_int64 * 33)()
        _check(lib().gko_matrix_plan(self.handle, C.byref(K), C.byref(S), C.byref(R), C.byref(cap), C.byref(thr),
                                     C.byref(nl), C.byref(nc), hist), "plan")
        return dict(kernel=K.value, subwarp=S.value, rows_per_subwarp=R.value, stage_cap=cap.value,
                    long_threshold=thr.value, n_long_rows=nl.value, n_long_chunks=nc.value, hist=list(hist))

    def set_plan(self, kernel: int, subwarp: int, rows_per_subwarp: int, stage_cap: int = 2048, stream=None):
        _check(lib().gko_matrix_set_plan(self.handle, kernel, subwarp, rows_per_subwarp, stage_cap,
                                         _stream(stream)), "set_plan")

    def tune(self, x, y, reps: int = 2, keep_kernel: bool = False, stream=None):
        """Time the candidate SpMV plans on device vectors x, y and keep the
        fastest (keep_kernel: only the current kernel's parameters); returns
        (kernel, subwarp, rows_per_subwarp, stage_cap, ms)."""
        k, S, R, cap = (C.c_int32() for _ in range(4))
        ms = C.c_float()
        _check(lib().gko_matrix_tune(self.handle, _dptr(x), _dptr(y), reps, 1 if keep_kernel else 0, C.byref(k),
                                     C.byref(S), C.byref(R), C.byref(cap), C.byref(ms), _stream(stream)),
               "gko_matrix_tune")
        return k.value, S.value, R.value, cap.value, ms.value

    def export(self, stream=None):
        """Host copies of the device arrays (dict of numpy arrays)."""
        inf = self.info()
        vdt = {F64: np.float64, F32: np.float32, BF16: np.uint16}[inf["dtype"]]
        out = {}
        args = [None] * 8
        if inf["format"] == CSR:
            out["row_ptr"] = np.empty(inf["n_rows"] + 1, np.int32)
            out["col"] = np.empty(inf["nnz"], np.int32)
            out["val"] = np.empty(inf["nnz"], vdt)
            args[0:3] = [out["row_ptr"], out["col"], out["val"]]
        if inf["format"] in (ELL, HYBRID):
            slots = inf["ell_width"] * inf["ell_stride"]
            out["ell_col"] = np.empty(slots, np.int32)
            out["ell_val"] = np.empty(slots, vdt)
            args[3:5] = [out["ell_col"], out["ell_val"]]
        if inf["format"] == SELLP:  # slice offsets in row_ptr, slots in ell_*
            n_slices = (inf["n_rows"] + inf["ell_stride"] - 1) // inf["ell_stride"]
            out["sets"] = np.empty(n_slices + 1, np.int32)
            out["ell_col"] = np.empty(inf["coo_nnz"], np.int32)
            out["ell_val"] = np.empty(inf["coo_nnz"], vdt)
            args[0] = out["sets"]
            args[3:5] = [out["ell_col"], out["ell_val"]]
        if inf["format"] in (COO, HYBRID):
            out["coo_row"] = np.empty(inf["coo_nnz"], np.int32)
            out["coo_col"] = np.empty(inf["coo_nnz"], np.int32)
            out["coo_val"] = np.empty(inf["coo_nnz"], vdt)
            args[5:8] = [out["coo_row"], out["coo_col"], out["coo_val"]]
        _check(lib().gko_matrix_export(self.handle, *[_hptr(a) for a in args], _stream(stream)), "export")
        out.update(inf)
        return out


def gko_matrix_create_csr(n_rows, n_cols, row_ptr, col, values, dtype=F64, stream=None) -> Matrix:
    """Create from host numpy arrays or device torch tensors."""
    h = C.c_void_p()
    on_dev = not isinstance(row_ptr, np.ndarray)
    if on_dev:
        nnz = int(col.numel())
        ptrs = (_dptr(row_ptr), _dptr(col), _dptr(values))
    else:
        row_ptr = np.ascontiguousarray(row_ptr, np.int32)
        col = np.ascontiguousarray(col, np.int32)
        values = np.ascontiguousarray(values)
        nnz = int(col.size)
        ptrs = (_hptr(row_ptr), _hptr(col), _hptr(values))
    _check(lib().gko_matrix_create_csr(n_rows, n_cols, nnz, *ptrs, dtype, 1 if on_dev else 0, _stream(stream),
                                       C.byref(h)), "gko_matrix_create_csr")
    return Matrix(h)


def from_csr(A, dtype=F64, stream=None) -> Matrix:
    """Create from an object with n_rows, n_cols, row_ptr, col, val (host)."""
    vals = np.ascontiguousarray(A.val, dtype=_NP_DTYPE.get(dtype, np.float64))
    if dtype == BF16:
        raise ValueError("create F64/F32 and convert with gko_matrix_convert_values for BF16")
    return gko_matrix_create_csr(A.n_rows, A.n_cols, A.row_ptr, A.col, vals, dtype, stream)


def _convert(fn, where, *args, stream=None) -> Matrix:
    h = C.c_void_p()
    _check(fn(*args, _stream(stream), C.byref(h)), where)
    return Matrix(h)


def gko_matrix_convert_to_ell(A: Matrix, max_fill: float = 0.0, stream=None) -> Matrix:
    return _convert(lib().gko_matrix_convert_to_ell, "convert_to_ell", A.handle, max_fill, stream=stream)


def gko_matrix_convert_to_coo(A: Matrix, stream=None) -> Matrix:
    return _convert(lib().gko_matrix_convert_to_coo, "convert_to_coo", A.handle, stream=stream)


def gko_matrix_convert_to_hybrid(A: Matrix, ell_width: int = -1, stream=None) -> Matrix:
    return _convert(lib().gko_matrix_convert_to_hybrid, "convert_to_hybrid", A.handle, ell_width, stream=stream)


def gko_matrix_convert_to_sellp(A: Matrix, slice_size: int = 0, max_fill: float = 0.0, stream=None) -> Matrix:
    return _convert(lib().gko_matrix_convert_to_sellp, "convert_to_sellp", A.handle, slice_size, max_fill,
                    stream=stream)


def gko_matrix_convert_values(A: Matrix, to: int, stream=None) -> Matrix:
    return _convert(lib().gko_matrix_convert_values, "convert_values", A.handle, to, stream=stream)


# ---------------------------------------------------------------------- SpMV

def gko_spmv(alpha: float, A: Matrix, x, beta: float, y, vec_dtype=None, stream=None):
    """y = alpha*A*x + beta*y on device tensors (asynchronous)."""
    import torch
    if vec_dtype is None:
        vec_dtype = F64 if y.dtype == torch.float64 else F32
    a, b = C.c_double(alpha), C.c_double(beta)
    _check(lib().gko_spmv(C.byref(a), A.handle, _dptr(x), C.byref(b), _dptr(y), vec_dtype, _stream(stream)),
           "gko_spmv")
    return y


def gko_spmv_host(alpha: float, A: Matrix, x_host, beta: float, y_host, x_dev, y_dev, stream=None):
    """y_host = alpha*A*x_host + beta*y_host through device buffers x_dev /
    y_dev (torch tensors; host ones pinned), stream-ordered, asynchronous."""
    import torch

    vdt = F64 if x_dev.dtype == torch.float64 else F32
    a, b = C.c_double(alpha), C.c_double(beta)
    _check(lib().gko_spmv_host(C.byref(a), A.handle, C.c_void_p(x_host.data_ptr()), C.byref(b),
                               C.c_void_p(y_host.data_ptr()), vdt, _dptr(x_dev), _dptr(y_dev), _stream(stream)),
           "gko_spmv_host")
    return y_host


def gko_spmv_coo_noalloc(alpha: float, A: Matrix, x, beta: float, y, stream=None):
    """y = alpha*A*x + beta*y for an F64 COO handle without any allocation."""
    a, b = C.c_double(alpha), C.c_double(beta)
    _check(lib().gko_spmv_coo_noalloc(C.byref(a), A.handle, _dptr(x), C.byref(b), _dptr(y), _stream(stream)),
           "gko_spmv_coo_noalloc")
    return y


SUBWARP_LIBRARY, SUBWARP_COOPERATIVE_GROUPS, SUBWARP_LEGACY = 0, 1, 2


def gko_bench_subwarp_reduce(subwarp: int, impl: int, data, inner_loops: int, stream=None):
    """Section 3.3 subwarp reduction benchmark on a float64/float32 CUDA
    tensor (length a multiple of 256), in place."""
    import torch

    dt = F64 if data.dtype == torch.float64 else F32
    _check(lib().gko_bench_subwarp_reduce(subwarp, impl, dt, inner_loops, _dptr(data), data.numel(),
                                          _stream(stream)), "gko_bench_subwarp_reduce")
    return data


def gko_bench_fma(data, inner_loops: int, stream=None):
    """FMA throughput probe on a float64/float32 CUDA tensor (length a
    multiple of 256), in place: 8 * numel * inner_loops FMAs."""
    import torch

    dt = F64 if data.dtype == torch.float64 else F32
    _check(lib().gko_bench_fma(dt, inner_loops, _dptr(data), data.numel(), _stream(stream)), "gko_bench_fma")
    return data


def gko_bench_gather(x, out, inner_loops: int, stream=None):
    """Random-gather probe: x a float64/float32 CUDA tensor of 2^k elements,
    out one element per thread of the same dtype (length a multiple of 256);
    8 * out.numel() * inner_loops gathers."""
    import torch

    n_x = x.numel()
    k = n_x.bit_length() - 1
    if n_x != 1 << k or out.dtype != x.dtype:
        raise ValueError("x needs a power-of-two length and out the same dtype")
    dt = F64 if x.dtype == torch.float64 else F32
    _check(lib().gko_bench_gather(dt, inner_loops, _dptr(x), k, _dptr(out), out.numel(), _stream(stream)),
           "gko_bench_gather")
    return out


def gko_diag_bounded_wait(cycles: int, stream=None) -> bool:
    """Run the bounded-wait failure check; True when the wait gave up."""
    t = C.c_int32()
    _check(lib().gko_diag_bounded_wait(cycles, C.byref(t), _stream(stream)), "gko_diag_bounded_wait")
    return bool(t.value)


def gko_dot(x, y, stream=None) -> float:
    r = C.c_double()
    _check(lib().gko_dot(x.numel(), _dptr(x), _dptr(y), C.byref(r), _stream(stream)), "gko_dot")
    return r.value


def gko_nrm2(x, stream=None) -> float:
    r = C.c_double()
    _check(lib().gko_nrm2(x.numel(), _dptr(x), C.byref(r), _stream(stream)), "gko_nrm2")
    return r.value


def gko_axpy(a: float, x, y, stream=None):
    _check(lib().gko_axpy(x.numel(), a, _dptr(x), _dptr(y), _stream(stream)), "gko_axpy")
    return y


def gko_multi_dot(V, w, k: int, stream=None) -> np.ndarray:
    """h[j] = V[j] . w for the first k rows of the 2-D tensor V."""
    h = np.empty(k, np.float64)
    _check(lib().gko_multi_dot(w.numel(), k, _dptr(V), V.stride(0), _dptr(w), _hptr(h), _stream(stream)),
           "gko_multi_dot")
    return h


def gko_multi_axpy_norm(V, h: np.ndarray, y, stream=None) -> float:
    """y -= sum_j h[j] V[j]; returns ||y||."""
    h = np.ascontiguousarray(h, np.float64)
    r = C.c_double()
    _check(lib().gko_multi_axpy_norm(y.numel(), h.size, _hptr(h), _dptr(V), V.stride(0), _dptr(y), C.byref(r),
                                     _stream(stream)), "gko_multi_axpy_norm")
    return r.value


def gko_spmv_dot(A: Matrix, x, y, stream=None) -> float:
    r = C.c_double()
    _check(lib().gko_spmv_dot(A.handle, _dptr(x), _dptr(y), C.byref(r), _stream(stream)), "gko_spmv_dot")
    return r.value


# ------------------------------------------------------------------- solvers

def _solve(name, A: Matrix, b, x, rel_tol, max_iters, opts=None, stream=None, raise_on_fail=False):
    fn = getattr(lib(), name, None)
    if fn is None:
        raise RuntimeError(f"{name} not available in {LIB_PATH}")
    res = SolveResult()
    st = fn(A.handle, _dptr(b), _dptr(x), rel_tol, max_iters, C.byref(opts) if opts is not None else None,
            C.byref(res), _stream(stream))
    if st not in (OK, NOT_CONVERGED, BREAKDOWN) or raise_on_fail:
        _check(st, name)
    return res


def gko_solve_cg(A, b, x, rel_tol=1e-10, max_iters=10000, opts=None, stream=None):
    return _solve("gko_solve_cg", A, b, x, rel_tol, max_iters, opts, stream)


def gko_solve_bicgstab(A, b, x, rel_tol=1e-10, max_iters=10000, opts=None, stream=None):
    return _solve("gko_solve_bicgstab", A, b, x, rel_tol, max_iters, opts, stream)


def gko_solve_gmres(A, b, x, rel_tol=1e-10, max_iters=10000, opts=None, stream=None):
    return _solve("gko_solve_gmres", A, b, x, rel_tol, max_iters, opts, stream)


PRECOND_NONE, PRECOND_JACOBI, PRECOND_BLOCK_JACOBI = 0, 1, 2


def gko_block_jacobi_inverse(A, block_size: int, B, stream=None) -> int:
    """Inverse diagonal blocks of an FP64 CSR handle into the device array B
    (n * block_size doubles, row i of its block's inverse at
    B[i*block_size:(i+1)*block_size]); returns how many blocks were singular
    (left as identity)."""
    sing = C.c_int64()
    _check(lib().gko_block_jacobi_inverse(A.handle, block_size, _dptr(B), C.byref(sing), _stream(stream)),
           "gko_block_jacobi_inverse")
    return int(sing.value)
BATCH_CSR, BATCH_ELL = 0, 1


def opts(restart=30, precision=PRECISION_F64, inner_tol=0.0, max_outer=0, inner_maxit=0, check_every=0,
         preconditioner=PRECOND_NONE, refinement=REFINE_AUTO, reliable_delta=0.0, block_size=0):
    return SolveOpts(restart, precision, inner_tol, max_outer, inner_maxit, check_every, preconditioner,
                     refinement, block_size, reliable_delta)


def gko_device_status(stream=None):
    """Raise if a kernel recorded a device-side failure (bounded wait timeout)."""
    _check(lib().gko_device_status(_stream(stream)), "gko_device_status")


class Batch:
    """Owning wrapper of a gko_batch handle (batched CG)."""

    def __init__(self, systems, storage=F64, stream=None):
        """systems: list of objects with n_rows, row_ptr, col, val (host CSR,
        FP64 values); the library concatenates them and, for F32 storage,
        rounds the values on the device."""
        count = len(systems)
        keep = [(np.ascontiguousarray(S.row_ptr, np.int32), np.ascontiguousarray(S.col, np.int32),
                 np.ascontiguousarray(S.val, np.float64)) for S in systems]
        n_rows = np.array([S.n_rows for S in systems], np.int32)
        rps = (C.c_void_p * count)(*[a[0].ctypes.data for a in keep])
        cols = (C.c_void_p * count)(*[a[1].ctypes.data for a in keep])
        vals = (C.c_void_p * count)(*[a[2].ctypes.data for a in keep])
        h = C.c_void_p()
        _check(lib().gko_batch_create_systems(count, _hptr(n_rows), rps, cols, vals, storage, _stream(stream),
                                              C.byref(h)), "gko_batch_create_systems")
        self.handle = h
        self.count = count
        self.storage = storage
        inf = self.info()
        self.total_rows = inf["total_rows"]
        self.total_nnz = inf["total_nnz"]
        self.row_off, self.nnz_off = self.offsets(stream)

    def offsets(self, stream=None):
        """The library's row and nonzero offsets of the systems (host arrays)."""
        ro = np.empty(self.count + 1, np.int64)
        no = np.empty(self.count + 1, np.int64)
        _check(lib().gko_batch_export(self.handle, _hptr(ro), _hptr(no), None, None, None, _stream(stream)),
               "gko_batch_export")
        return ro, no

    def export(self, stream=None):
        """The stored arrays (row_off, nnz_off, row_ptr, col, values) on the host."""
        ro = np.empty(self.count + 1, np.int64)
        no = np.empty(self.count + 1, np.int64)
        rp = np.empty(self.total_rows + self.count, np.int32)
        col = np.empty(self.total_nnz, np.int32)
        val = np.empty(self.total_nnz, np.float64 if self.storage == F64 else np.float32)
        _check(lib().gko_batch_export(self.handle, _hptr(ro), _hptr(no), _hptr(rp), _hptr(col), _hptr(val),
                                      _stream(stream)), "gko_batch_export")
        return ro, no, rp, col, val

    def __del__(self):
        try:
            if self.handle and _lib is not None:
                _lib.gko_batch_destroy(self.handle)
        except Exception:
            pass
        self.handle = None

    def cg(self, b, x, rel_tol=1e-10, max_iters=10000, stream=None):
        it = np.zeros(self.count, np.int32)
        rr = np.zeros(self.count, np.float64)
        st = np.zeros(self.count, np.int32)
        code = lib().gko_batch_cg(self.handle, _dptr(b), _dptr(x), rel_tol, max_iters, _hptr(it), _hptr(rr),
                                  _hptr(st), _stream(stream))
        if code not in (OK, NOT_CONVERGED, BREAKDOWN):
            _check(code, "gko_batch_cg")
        return code, it, rr, st

    def tune(self, b, x0, rel_tol=1e-10, max_iters=10000, stream=None):
        """The autotuner: returns dict(warp_rows, threads, storage, ms)."""
        wr, th, st = C.c_int32(), C.c_int32(), C.c_int32()
        ms = C.c_float()
        _check(lib().gko_batch_tune(self.handle, _dptr(b), _dptr(x0), rel_tol, max_iters, C.byref(wr), C.byref(th),
                                    C.byref(st), C.byref(ms), _stream(stream)), "gko_batch_tune")
        return dict(warp_rows=wr.value, threads=th.value, storage="ell" if st.value == BATCH_ELL else "csr",
                    ms=round(ms.value, 3))

    def set_threshold(self, warp_rows, stream=None):
        _check(lib().gko_batch_set_threshold(self.handle, warp_rows, _stream(stream)), "gko_batch_set_threshold")

    def set_precision(self, precision, reliable_delta=0.0, stream=None):
        """PRECISION_F64, or PRECISION_MIXED_F32 (reliable-update CG per system)."""
        _check(lib().gko_batch_set_precision(self.handle, precision, reliable_delta, _stream(stream)),
               "gko_batch_set_precision")

    def last_updates(self, stream=None):
        up = np.zeros(self.count, np.int32)
        _check(lib().gko_batch_last_updates(self.handle, up.ctypes.data_as(_P), _stream(stream)),
               "gko_batch_last_updates")
        return up

    def set_schedule(self, warp_rows, threads=256, storage=None, stream=None):
        st = BATCH_CSR if storage is None else storage
        _check(lib().gko_batch_set_schedule(self.handle, warp_rows, threads, st, _stream(stream)),
               "gko_batch_set_schedule")

    def info(self):
        c, wr, ni, th, st = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        tr, tn = C.c_int64(), C.c_int64()
        _check(lib().gko_batch_info(self.handle, C.byref(c), C.byref(tr), C.byref(tn), C.byref(wr), C.byref(ni),
                                    C.byref(th), C.byref(st)), "gko_batch_info")
        return dict(count=c.value, total_rows=tr.value, total_nnz=tn.value, warp_rows=wr.value, n_items=ni.value,
                    threads=th.value, storage="ell" if st.value == BATCH_ELL else "csr")


class Server:
    """Owning wrapper of a gko_server (continuous-batching request loop)."""

    def __init__(self, slots=4, budget_bytes=0):
        h = C.c_void_p()
        _check(lib().gko_server_create(slots, int(budget_bytes), C.byref(h)), "gko_server_create")
        self.handle = h
        self._mats = []
        self._n = {}

    def add_matrix(self, M: Matrix) -> int:
        mid = C.c_int32()
        _check(lib().gko_server_add_matrix(self.handle, M.handle, C.byref(mid)), "gko_server_add_matrix")
        self._mats.append(M)
        self._n[mid.value] = M.info()["n_rows"]
        return mid.value

    def submit(self, matrix_id: int, solver: int, b: np.ndarray, rel_tol=1e-8, max_iters=1000, opts=None) -> int:
        b = np.ascontiguousarray(b, np.float64)
        rid = C.c_int64()
        _check(lib().gko_server_submit(self.handle, matrix_id, solver, _hptr(b), rel_tol, max_iters,
                                       C.byref(opts) if opts is not None else None, C.byref(rid)), "gko_server_submit")
        self._pending = getattr(self, "_pending", {})
        self._pending[rid.value] = self._n[matrix_id]
        return rid.value

    def result(self, request_id: int, wait=True):
        """(status, SolveResult, x, latency_ms) or None while still running."""
        n = self._pending.get(request_id, 0)
        x = np.empty(n, np.float64)
        done = C.c_int32()
        res = SolveResult()
        lat = C.c_double()
        st = lib().gko_server_result(self.handle, request_id, 1 if wait else 0, C.byref(done), C.byref(res),
                                     _hptr(x), C.byref(lat))
        if not done.value:
            if st != OK:
                _check(st, "gko_server_result")
            return None
        self._pending.pop(request_id, None)
        if st not in (OK, NOT_CONVERGED, BREAKDOWN):
            _check(st, "gko_server_result")
        return st, res, x, lat.value

    def stats(self):
        c = C.c_int64()
        p50, p99, sps = C.c_double(), C.c_double(), C.c_double()
        pk = C.c_int32()
        _check(lib().gko_server_stats(self.handle, C.byref(c), C.byref(p50), C.byref(p99), C.byref(sps),
                                      C.byref(pk)), "gko_server_stats")
        return dict(completed=c.value, p50_ms=p50.value, p99_ms=p99.value, solves_per_s=sps.value,
                    peak_active=pk.value)

    def close(self):
        if self.handle and _lib is not None:
            _lib.gko_server_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_memory_budget(nbytes: int):
    _check(lib().gko_set_memory_budget(int(nbytes)), "set_memory_budget")


def memory_in_use() -> int:
    v = C.c_int64()
    _check(lib().gko_memory_in_use(C.byref(v)), "memory_in_use")
    return v.value
