"""Plain FP64 CPU oracle for the sparse hot path -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it.

The arithmetic lives in ``gko_oracle.c`` (plain sequential C, FP64, no FMA
contraction); this module only marshals numpy arrays into it.  See the C file
header for the definitions followed (the paper's format and solver list in
Section 1, with textbook algorithms: Bell & Garland SC'09 for the formats,
Saad's "Iterative Methods for Sparse Linear Systems" for CG, BiCGSTAB and
GMRES, Buttari et al. 2007 for mixed-precision refinement).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from .build import build as _build, lib_path

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None

CG, BICGSTAB, GMRES = 0, 1, 2
STATUS_OK, STATUS_NOT_CONVERGED, STATUS_BREAKDOWN = 0, 4, 5


class _Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32),
                ("outer_iterations", C.c_int32), ("pad", C.c_int32),
                ("rel_residual", C.c_double)]


@dataclass
class SolveResult:
    status: int
    iterations: int
    outer_iterations: int
    rel_residual: float


_P = C.c_void_p
_I64 = C.c_int64
_I32 = C.c_int32
_D = C.c_double
_F = C.c_float

_SIGS = {
    "or_set_threads": (C.c_int, [C.c_int]),
    "or_has_openmp": (C.c_int, []),
    "or_spmv_csr": (None, [_I64, _P, _P, _P, _P, _D, _D, _P]),
    "or_spmv_csr_f32": (None, [_I64, _P, _P, _P, _P, _F, _F, _P]),
    "or_spmv_csr_exact": (None, [_I64, _P, _P, _P, _P, _D, _D, _P]),
    "or_ell_stride": (_I64, [_I64]),
    "or_ell_width": (_I32, [_I64, _P]),
    "or_csr_to_ell": (None, [_I64, _P, _P, _P, _I32, _I64, _P, _P]),
    "or_spmv_ell": (None, [_I64, _I32, _I64, _P, _P, _P, _D, _D, _P]),
    "or_sellp_slices": (_I64, [_I64, _I32]),
    "or_sellp_sets": (_I64, [_I64, _P, _I32, _P]),
    "or_csr_to_sellp": (None, [_I64, _P, _P, _P, _I32, _P, _P, _P]),
    "or_spmv_sellp": (None, [_I64, _I32, _P, _P, _P, _P, _D, _D, _P]),
    "or_subwarp_reduce": (None, [_I64, _I32, _I32, _P]),
    "or_csr_to_coo": (None, [_I64, _P, _P, _P, _P, _P, _P]),
    "or_spmv_coo": (C.c_int, [_I64, _I64, _P, _P, _P, _P, _D, _D, _P]),
    "or_hybrid_width": (_I32, [_I64, _P]),
    "or_hybrid_tail_nnz": (_I64, [_I64, _P, _I32]),
    "or_csr_to_hybrid": (None, [_I64, _P, _P, _P, _I32, _I64, _P, _P, _P, _P, _P]),
    "or_spmv_hybrid": (C.c_int, [_I64, _I32, _I64, _P, _P, _I64, _P, _P, _P, _P, _D, _D, _P]),
    "or_dot": (_D, [_I64, _P, _P]),
    "or_axpy": (None, [_I64, _D, _P, _P]),
    "or_multi_dot": (None, [_I64, _I32, _P, _I64, _P, _P]),
    "or_multi_axpy_norm": (_D, [_I64, _I32, _P, _P, _I64, _P]),
    "or_solve": (C.c_int, [C.c_int, _I64, _P, _P, _P, _P, _P, _D, _I32, _I32, _P, _I32,
                           C.POINTER(_Result)]),
    "or_solve_ir": (C.c_int, [C.c_int, _I64, _P, _P, _P, _P, _P, _P, _D, _I32, _D, _I32, _I32, _I32,
                              C.POINTER(_Result)]),
    "or_jacobi_inv": (None, [_I64, _P, _P, _P, _P]),
    "or_block_jacobi_inv": (_I64, [_I64, _P, _P, _P, _I32, _P]),
    "or_solve_bj": (C.c_int, [C.c_int, _I64, _P, _P, _P, _I32, _P, _P, _P, _D, _I32, C.POINTER(_Result)]),
    "or_solve_ir_bj": (C.c_int, [C.c_int, _I64, _P, _P, _P, _P, _I32, _P, _P, _P, _D, _I32, _D, _I32, _I32,
                                 C.POINTER(_Result)]),
    "or_solve_reliable_bj": (C.c_int, [C.c_int, _I64, _P, _P, _P, _P, _I32, _P, _I32, _P, _P, _D, _I32, _D,
                                       C.POINTER(_Result)]),
    "or_batch_cg": (None, [_I32, _P, _P, _P, _P, _P, _P, _P, _D, _I32, _P, _P, _P]),
    "or_solve_pc": (C.c_int, [C.c_int, _I64, _P, _P, _P, _P, _P, _P, _D, _I32, C.POINTER(_Result)]),
    "or_solve_ir_pc": (C.c_int, [C.c_int, _I64, _P, _P, _P, _P, _P, _P, _P, _D, _I32, _D, _I32, _I32,
                                 C.POINTER(_Result)]),
    "or_solve_reliable": (C.c_int, [C.c_int, _I64, _P, _P, _P, _P, _P, _I32, _P, _P, _D, _I32, _D,
                                    C.POINTER(_Result)]),
    "or_batch_cg_reliable": (None, [_I32, _P, _P, _P, _P, _P, _P, _P, _P, _D, _I32, _D, _P, _P, _P, _P]),
}


def lib():
    """Load (building on first use) the oracle shared library."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            _build()
        L = C.CDLL(path)
        for name, (ret, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = ret
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(t: int) -> int:
    """Threads for the row-parallel CSR/ELL SpMV loops; returns the count used."""
    return int(lib().or_set_threads(int(t)))


def has_openmp() -> bool:
    return bool(lib().or_has_openmp())


def _y0(n, y, beta, dtype=np.float64):
    if y is None:
        return np.zeros(n, dtype=dtype)
    return np.array(y, dtype=dtype, copy=True)


def spmv_csr(A, x, alpha=1.0, beta=0.0, y=None):
    """y = alpha*A*x + beta*y (FP64, sequential row sums in storage order)."""
    rp, col, val, x = _i32(A.row_ptr), _i32(A.col), _f64(A.val), _f64(x)
    out = _y0(A.n_rows, y, beta)
    lib().or_spmv_csr(A.n_rows, _p(rp), _p(col), _p(val), _p(x), alpha, beta, _p(out))
    return out


def spmv_csr_f32(A, x, alpha=1.0, beta=0.0, y=None):
    """FP32 values/x/y with FP32 accumulation (each product and sum rounded)."""
    rp, col = _i32(A.row_ptr), _i32(A.col)
    val = np.ascontiguousarray(A.val, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = _y0(A.n_rows, y, beta, np.float32)
    lib().or_spmv_csr_f32(A.n_rows, _p(rp), _p(col), _p(val), _p(x), alpha, beta, _p(out))
    return out


def spmv_csr_exact(A, x, alpha=1.0, beta=0.0, y=None):
    """Compensated (TwoSum/TwoProduct, Neumaier) row sums: near-exact y."""
    rp, col, val, x = _i32(A.row_ptr), _i32(A.col), _f64(A.val), _f64(x)
    out = _y0(A.n_rows, y, beta)
    lib().or_spmv_csr_exact(A.n_rows, _p(rp), _p(col), _p(val), _p(x), alpha, beta, _p(out))
    return out


def spmv_abs_scale(A, x, alpha=1.0, beta=0.0, y=None):
    """s_i = |alpha| * sum_k |a_ik x_ck| + |beta y_i|: the componentwise scale
    against which a reordered FP sum is judged."""
    absA = type(A)(A.n_rows, A.n_cols, A.row_ptr, A.col, np.abs(_f64(A.val)), A.name)
    s = spmv_csr(absA, np.abs(_f64(x)), abs(alpha), 0.0)
    if y is not None and beta != 0.0:
        s = s + abs(beta) * np.abs(_f64(y))
    return s


@dataclass
class Ell:
    n_rows: int
    K: int
    stride: int
    col: np.ndarray  # int32[K*stride]
    val: np.ndarray  # float64[K*stride]


def ell_stride(n: int) -> int:
    return int(lib().or_ell_stride(n))


def ell_width(A) -> int:
    return int(lib().or_ell_width(A.n_rows, _p(_i32(A.row_ptr))))


def csr_to_ell(A, K=None) -> Ell:
    rp, col, val = _i32(A.row_ptr), _i32(A.col), _f64(A.val)
    if K is None:
        K = ell_width(A)
    stride = ell_stride(A.n_rows)
    ecol = np.empty(K * stride, np.int32)
    eval_ = np.empty(K * stride, np.float64)
    lib().or_csr_to_ell(A.n_rows, _p(rp), _p(col), _p(val), K, stride, _p(ecol), _p(eval_))
    return Ell(A.n_rows, K, stride, ecol, eval_)


def spmv_ell(E: Ell, x, alpha=1.0, beta=0.0, y=None):
    x = _f64(x)
    out = _y0(E.n_rows, y, beta)
    lib().or_spmv_ell(E.n_rows, E.K, E.stride, _p(E.col), _p(E.val), _p(x), alpha, beta, _p(out))
    return out


def subwarp_reduce(data, S: int, loops: int):
    """Section 3.3 reduce benchmark: `loops` butterfly reductions over
    subwarps of S consecutive lanes; returns the lanes' final values."""
    d = _f64(data).copy()
    lib().or_subwarp_reduce(d.size, S, loops, _p(d))
    return d


@dataclass
class Sellp:
    n_rows: int
    C: int            # slice height
    sets: np.ndarray  # int64[n_slices+1], prefix sums of the slice widths
    col: np.ndarray   # int32[sets[-1]*C]
    val: np.ndarray   # float64[sets[-1]*C]


def csr_to_sellp(A, C=64) -> Sellp:
    """SELL-P (Section 1 Sellp; Anzt, Tomov & Dongarra 2014 layout): slices of
    C rows, each as wide as its longest row, column-major within the slice."""
    rp, col, val = _i32(A.row_ptr), _i32(A.col), _f64(A.val)
    ns = int(lib().or_sellp_slices(A.n_rows, C))
    sets = np.empty(ns + 1, np.int64)
    total = int(lib().or_sellp_sets(A.n_rows, _p(rp), C, _p(sets)))
    scol = np.empty(total * C, np.int32)
    sval = np.empty(total * C, np.float64)
    lib().or_csr_to_sellp(A.n_rows, _p(rp), _p(col), _p(val), C, _p(sets), _p(scol), _p(sval))
    return Sellp(A.n_rows, C, sets, scol, sval)


def spmv_sellp(S: Sellp, x, alpha=1.0, beta=0.0, y=None):
    x = _f64(x)
    out = _y0(S.n_rows, y, beta)
    lib().or_spmv_sellp(S.n_rows, S.C, _p(S.sets), _p(S.col), _p(S.val), _p(x), alpha, beta, _p(out))
    return out


@dataclass
class Coo:
    n_rows: int
    row: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self):
        return int(self.row.size)


def csr_to_coo(A) -> Coo:
    rp, col, val = _i32(A.row_ptr), _i32(A.col), _f64(A.val)
    nnz = int(rp[-1])
    r = np.empty(nnz, np.int32)
    c = np.empty(nnz, np.int32)
    v = np.empty(nnz, np.float64)
    lib().or_csr_to_coo(A.n_rows, _p(rp), _p(col), _p(val), _p(r), _p(c), _p(v))
    return Coo(A.n_rows, r, c, v)


def spmv_coo(M: Coo, x, alpha=1.0, beta=0.0, y=None):
    x = _f64(x)
    out = _y0(M.n_rows, y, beta)
    rc = lib().or_spmv_coo(M.n_rows, M.nnz, _p(_i32(M.row)), _p(_i32(M.col)), _p(_f64(M.val)),
                           _p(x), alpha, beta, _p(out))
    assert rc == 0
    return out


@dataclass
class Hybrid:
    ell: Ell
    coo: Coo


def hybrid_width(A) -> int:
    return int(lib().or_hybrid_width(A.n_rows, _p(_i32(A.row_ptr))))


def csr_to_hybrid(A, K=None) -> Hybrid:
    rp, col, val = _i32(A.row_ptr), _i32(A.col), _f64(A.val)
    if K is None or K < 0:
        K = hybrid_width(A)
    stride = ell_stride(A.n_rows)
    tail = int(lib().or_hybrid_tail_nnz(A.n_rows, _p(rp), K))
    ecol = np.empty(K * stride, np.int32)
    eval_ = np.empty(K * stride, np.float64)
    r = np.empty(tail, np.int32)
    c = np.empty(tail, np.int32)
    v = np.empty(tail, np.float64)
    lib().or_csr_to_hybrid(A.n_rows, _p(rp), _p(col), _p(val), K, stride, _p(ecol), _p(eval_),
                           _p(r), _p(c), _p(v))
    return Hybrid(Ell(A.n_rows, K, stride, ecol, eval_), Coo(A.n_rows, r, c, v))


def spmv_hybrid(H: Hybrid, x, alpha=1.0, beta=0.0, y=None):
    x = _f64(x)
    out = _y0(H.ell.n_rows, y, beta)
    E, M = H.ell, H.coo
    rc = lib().or_spmv_hybrid(E.n_rows, E.K, E.stride, _p(E.col), _p(E.val), M.nnz,
                              _p(_i32(M.row)), _p(_i32(M.col)), _p(_f64(M.val)), _p(x),
                              alpha, beta, _p(out))
    assert rc == 0
    return out


def dot(x, y) -> float:
    """Sequential FP64 dot product."""
    x, y = _f64(x), _f64(y)
    return float(lib().or_dot(x.size, _p(x), _p(y)))


def axpy(a, x, y):
    x = _f64(x)
    out = np.array(y, dtype=np.float64, copy=True)
    lib().or_axpy(x.size, a, _p(x), _p(out))
    return out


def multi_dot(V, w):
    """h_j = V[j] . w for each row of the 2-D array V."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    w = _f64(w)
    h = np.empty(V.shape[0])
    lib().or_multi_dot(w.size, V.shape[0], _p(V), V.shape[1], _p(w), _p(h))
    return h


def multi_axpy_norm(V, h, y):
    """Returns (y - sum_j h_j V[j], its 2-norm)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    h = _f64(h)
    out = np.array(y, dtype=np.float64, copy=True)
    nrm = lib().or_multi_axpy_norm(out.size, h.size, _p(h), _p(V), V.shape[1], _p(out))
    return out, float(nrm)


def solve(solver: int, A, b, x0=None, tol=1e-10, maxit=1000, restart=30, history=False):
    """FP64 CG / BiCGSTAB / GMRES(restart).  Returns (x, SolveResult[, hist])."""
    rp, col, val, b = _i32(A.row_ptr), _i32(A.col), _f64(A.val), _f64(b)
    x = np.zeros(A.n_rows) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    hist = np.full(max(maxit, 1), np.nan) if history else None
    res = _Result()
    lib().or_solve(solver, A.n_rows, _p(rp), _p(col), _p(val), _p(b), _p(x), tol, maxit, restart,
                   _p(hist) if hist is not None else None, maxit if history else 0, C.byref(res))
    out = SolveResult(res.status, res.iterations, res.outer_iterations, res.rel_residual)
    if history:
        return x, out, hist[: res.iterations]
    return x, out


def cg(A, b, **kw):
    return solve(CG, A, b, **kw)


def bicgstab(A, b, **kw):
    return solve(BICGSTAB, A, b, **kw)


def gmres(A, b, **kw):
    return solve(GMRES, A, b, **kw)


def solve_ir(solver: int, A, b, x0=None, tol=1e-8, max_outer=30, inner_tol=1e-4,
             inner_maxit=1000, restart=30, jacobi=False, adaptive=False, block_size=0):
    """Mixed-precision iterative refinement (FP32-stored inner solve, FP64
    outer); each inner solve reduces the residual by inner_tol (adaptive: by
    max(inner_tol, min(0.5, 0.5 tol ||b|| / ||r||)), the library's tunable);
    jacobi: the inner CG / BiCGSTAB is Jacobi preconditioned; block_size > 0:
    block-Jacobi with blocks of that size (inverse blocks rounded to FP32)."""
    rp, col, val, b = _i32(A.row_ptr), _i32(A.col), _f64(A.val), _f64(b)
    val32 = val.astype(np.float32)
    x = np.zeros(A.n_rows) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    res = _Result()
    if block_size:
        B, _ = block_jacobi_inv(A, block_size)
        lib().or_solve_ir_bj(solver, A.n_rows, _p(rp), _p(col), _p(val), _p(val32), block_size, _p(B), _p(b),
                             _p(x), tol, max_outer, inner_tol, inner_maxit, int(adaptive), C.byref(res))
    elif jacobi:
        minv = jacobi_inv(A)
        lib().or_solve_ir_pc(solver, A.n_rows, _p(rp), _p(col), _p(val), _p(val32), _p(minv), _p(b), _p(x),
                             tol, max_outer, inner_tol, inner_maxit, int(adaptive), C.byref(res))
    else:
        lib().or_solve_ir(solver, A.n_rows, _p(rp), _p(col), _p(val), _p(val32), _p(b), _p(x), tol,
                          max_outer, inner_tol, inner_maxit, restart, int(adaptive), C.byref(res))
    return x, SolveResult(res.status, res.iterations, res.outer_iterations, res.rel_residual)


def solve_reliable(solver: int, A, b, x0=None, tol=1e-8, maxit=5000, delta=0.1, f32=True, jacobi=False,
                   block_size=0):
    """CG / BiCGSTAB with reliable updates: recurrences on FP32 values with
    FP32-stored vectors (f32=False: the FP64 matrix and FP64 vectors), the
    partial solution folded into the FP64 x and the recurrence residual
    replaced by the FP64 residual b - A x whenever the recurrence residual
    meets tol ||b|| or drops below delta times its largest value since the
    last update.  outer_iterations counts the updates.  jacobi / block_size
    > 0: Jacobi / block-Jacobi preconditioned recurrences.  Returns (x,
    SolveResult)."""
    rp, col, val, b = _i32(A.row_ptr), _i32(A.col), _f64(A.val), _f64(b)
    val32 = val.astype(np.float32) if f32 else None
    if block_size:
        B, _ = block_jacobi_inv(A, block_size)
        x = np.zeros(A.n_rows) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        res = _Result()
        lib().or_solve_reliable_bj(solver, A.n_rows, _p(rp), _p(col), _p(val), _p(val32) if f32 else None,
                                   block_size, _p(B), int(bool(f32)), _p(b), _p(x), tol, maxit, delta,
                                   C.byref(res))
        return x, SolveResult(res.status, res.iterations, res.outer_iterations, res.rel_residual)
    minv = jacobi_inv(A) if jacobi else None
    x = np.zeros(A.n_rows) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    res = _Result()
    lib().or_solve_reliable(solver, A.n_rows, _p(rp), _p(col), _p(val), _p(val32) if f32 else None,
                            _p(minv) if jacobi else None, int(bool(f32)), _p(b), _p(x), tol, maxit, delta,
                            C.byref(res))
    return x, SolveResult(res.status, res.iterations, res.outer_iterations, res.rel_residual)


def jacobi_inv(A):
    """Inverse diagonal (diagonal entries of a row summed; zero -> 1)."""
    rp, col, val = _i32(A.row_ptr), _i32(A.col), _f64(A.val)
    out = np.empty(A.n_rows)
    lib().or_jacobi_inv(A.n_rows, _p(rp), _p(col), _p(val), _p(out))
    return out


def solve_jacobi(solver: int, A, b, x0=None, tol=1e-10, maxit=1000):
    """Jacobi-preconditioned FP64 CG (Saad Alg. 9.1) or right-preconditioned
    BiCGSTAB.  Returns (x, SolveResult)."""
    rp, col, val, b = _i32(A.row_ptr), _i32(A.col), _f64(A.val), _f64(b)
    minv = jacobi_inv(A)
    x = np.zeros(A.n_rows) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    res = _Result()
    lib().or_solve_pc(solver, A.n_rows, _p(rp), _p(col), _p(val), _p(minv), _p(b), _p(x), tol, maxit,
                      C.byref(res))
    return x, SolveResult(res.status, res.iterations, res.outer_iterations, res.rel_residual)


def block_jacobi_inv(A, bs: int):
    """Inverse diagonal blocks of size bs (rows k*bs .. k*bs + nb - 1, the
    last block possibly smaller), each by Gauss-Jordan elimination with
    partial pivoting; a singular block becomes the identity.  Returns
    (B, singular): B[i, j] = row i of its block's inverse at column j of the
    block (zeros past the last block's size), singular = blocks replaced."""
    rp, col, val = _i32(A.row_ptr), _i32(A.col), _f64(A.val)
    B = np.empty((A.n_rows, bs))
    singular = lib().or_block_jacobi_inv(A.n_rows, _p(rp), _p(col), _p(val), bs, _p(B))
    if singular < 0:
        raise ValueError("block size must lie in 1..64")
    return B, int(singular)


def solve_block_jacobi(solver: int, A, b, bs: int, x0=None, tol=1e-10, maxit=1000):
    """Block-Jacobi-preconditioned FP64 CG (Saad Alg. 9.1 with M the block
    diagonal of A) or right-preconditioned BiCGSTAB.  Returns (x, SolveResult)."""
    rp, col, val, b = _i32(A.row_ptr), _i32(A.col), _f64(A.val), _f64(b)
    B, _ = block_jacobi_inv(A, bs)
    x = np.zeros(A.n_rows) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    res = _Result()
    lib().or_solve_bj(solver, A.n_rows, _p(rp), _p(col), _p(val), bs, _p(B), _p(b), _p(x), tol, maxit,
                      C.byref(res))
    return x, SolveResult(res.status, res.iterations, res.outer_iterations, res.rel_residual)


def batch_cg(systems, bs, x0=None, tol=1e-10, maxit=10000):
    """The single-system CG on every system of a batch (OpenMP over systems).
    systems: list of host CSR objects; bs: right-hand sides.  Returns
    (x per system, iterations, true relative residuals, statuses)."""
    count = len(systems)
    rows = np.array([S.n_rows for S in systems], np.int64)
    nnzs = np.array([int(S.row_ptr[-1]) for S in systems], np.int64)
    row_off = np.concatenate([[0], np.cumsum(rows)]).astype(np.int64)
    nnz_off = np.concatenate([[0], np.cumsum(nnzs)]).astype(np.int64)
    rp = np.concatenate([_i32(S.row_ptr) for S in systems])
    col = np.concatenate([_i32(S.col) for S in systems])
    val = np.concatenate([_f64(S.val) for S in systems])
    b = np.concatenate([_f64(v) for v in bs])
    x = np.zeros(b.size) if x0 is None else np.concatenate([_f64(v) for v in x0])
    it = np.zeros(count, np.int32)
    rr = np.zeros(count, np.float64)
    st = np.zeros(count, np.int32)
    lib().or_batch_cg(count, _p(row_off), _p(nnz_off), _p(rp), _p(col), _p(val), _p(b), _p(x), tol, maxit,
                      _p(it), _p(rr), _p(st))
    return [x[row_off[i]:row_off[i + 1]] for i in range(count)], it, rr, st


def batch_cg_reliable(systems, bs, x0=None, tol=1e-10, maxit=10000, delta=0.1, storage_f32=False):
    """The single-system reliable-update CG on every system of a batch
    (OpenMP over systems): recurrences on the systems' FP32 values, replaced
    residuals with their FP64 values (storage_f32: the systems are their
    FP32 roundings, so both use those).  Returns (x per system, iterations,
    updates, true relative residuals, statuses)."""
    count = len(systems)
    rows = np.array([S.n_rows for S in systems], np.int64)
    nnzs = np.array([int(S.row_ptr[-1]) for S in systems], np.int64)
    row_off = np.concatenate([[0], np.cumsum(rows)]).astype(np.int64)
    nnz_off = np.concatenate([[0], np.cumsum(nnzs)]).astype(np.int64)
    rp = np.concatenate([_i32(S.row_ptr) for S in systems])
    col = np.concatenate([_i32(S.col) for S in systems])
    val = np.concatenate([_f64(S.val) for S in systems])
    val32 = val.astype(np.float32)
    if storage_f32:
        val = val32.astype(np.float64)
    b = np.concatenate([_f64(v) for v in bs])
    x = np.zeros(b.size) if x0 is None else np.concatenate([_f64(v) for v in x0])
    it = np.zeros(count, np.int32)
    up = np.zeros(count, np.int32)
    rr = np.zeros(count, np.float64)
    st = np.zeros(count, np.int32)
    lib().or_batch_cg_reliable(count, _p(row_off), _p(nnz_off), _p(rp), _p(col), _p(val), _p(val32), _p(b), _p(x),
                               tol, maxit, delta, _p(it), _p(up), _p(rr), _p(st))
    return [x[row_off[i]:row_off[i + 1]] for i in range(count)], it, up, rr, st
