"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module builds test matrices and vectors only; it contains none of the
method's arithmetic (no SpMV, no dot products, no solver steps).  Every matrix
is returned as plain CSR arrays (int32 ``row_ptr``/``col``, float64 ``val``)
in natural lexicographic order ``idx = i + N*(j + N*k)`` with ``i`` fastest.

Matrix families (the workload classes named by the paper's evaluation,
Section 4, which used SuiteSparse matrices; synthetic stand-ins are used here):

* ``laplace2d_5pt``   2D 5-point Laplacian, Dirichlet by truncation, diag 4, off -1
* ``stencil3d_7pt``   3D 7-point Laplacian, diag 6, off -1
* ``stencil3d_27pt``  3D 27-point stencil, diag 26, off -1
* ``convdiff3d_7pt``  3D 7-point upwind convection-diffusion with cell Peclet P:
                      diag 6+3P, upstream (-x,-y,-z) neighbours -1-P, downstream -1
* ``varcoef2d_5pt`` / ``varcoef3d_7pt``  variable-coefficient diffusion: cell
                      coefficients exp(N(0,1)), face = harmonic mean of the two
                      cells, a Dirichlet boundary face uses the cell's own value,
                      off-diagonal = -face, diagonal = sum of the cell's faces
* ``powerlaw``        row lengths Zipf(s=2) clipped to [1, 10000] (optionally
                      scaled by lambda before clipping), uniform random columns
                      (unsorted, duplicates allowed), values N(0,1)
* ``banded``          diagonal always present, each off-diagonal slot within the
                      half-bandwidth present with probability p, values U[-1,1]

Random numbers come from numpy's PCG64 ``default_rng``; the draw order of each
generator is fixed and documented in its docstring.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Csr:
    """Plain host CSR arrays (int32 indices, float64 values)."""

    n_rows: int
    n_cols: int
    row_ptr: np.ndarray  # int32[n_rows + 1]
    col: np.ndarray  # int32[nnz]
    val: np.ndarray  # float64[nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))


def _assemble(n: int, cols: np.ndarray, vals: np.ndarray, valid: np.ndarray, name: str) -> Csr:
    """Pack (n, S) candidate slots into CSR, keeping slot order within a row."""
    counts = valid.sum(axis=1, dtype=np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 indices")
    return Csr(n, n, row_ptr.astype(np.int32), np.ascontiguousarray(cols[valid], dtype=np.int32),
               np.ascontiguousarray(vals[valid], dtype=np.float64), name)


def _coords(shape):
    n = int(np.prod(shape))
    idx = np.arange(n, dtype=np.int64)
    out = []
    for s in shape:
        out.append((idx % s).astype(np.int32))
        idx //= s
    return n, out


def _stencil(shape, offsets, weight) -> tuple:
    """Candidate slots for a constant stencil: offsets sorted by linear offset."""
    n, coords = _coords(shape)
    strides = [int(np.prod(shape[:a])) for a in range(len(shape))]
    lin = np.arange(n, dtype=np.int64)
    S = len(offsets)
    cols = np.empty((n, S), dtype=np.int32)
    vals = np.empty((n, S), dtype=np.float64)
    valid = np.empty((n, S), dtype=bool)
    for s, off in enumerate(offsets):
        ok = np.ones(n, dtype=bool)
        shift = 0
        for a, d in enumerate(off):
            if d:
                c = coords[a] + d
                ok &= (c >= 0) & (c < shape[a])
                shift += d * strides[a]
        valid[:, s] = ok
        cols[:, s] = np.where(ok, lin + shift, 0)
        vals[:, s] = weight(off)
    return n, cols, vals, valid


def _sorted_offsets(dim, full):
    if full:
        grid = np.array(np.meshgrid(*([[-1, 0, 1]] * dim), indexing="ij")).reshape(dim, -1).T
        offs = [tuple(int(v) for v in o) for o in grid]
    else:
        offs = [tuple(0 for _ in range(dim))]
        for a in range(dim):
            for d in (-1, 1):
                o = [0] * dim
                o[a] = d
                offs.append(tuple(o))
    # ascending linear offset (i fastest) gives ascending column order in a row
    def lin(o):
        return sum(d * (10 ** (3 * a)) for a, d in enumerate(o))
    return sorted(offs, key=lin)


def laplace2d_5pt(N: int) -> Csr:
    """2D 5-point Laplacian on an N x N grid: diag 4, neighbours -1."""
    offs = _sorted_offsets(2, False)
    n, cols, vals, valid = _stencil((N, N), offs, lambda o: 4.0 if not any(o) else -1.0)
    return _assemble(n, cols, vals, valid, f"laplace2d_5pt_{N}")


def stencil3d_7pt(N: int) -> Csr:
    """3D 7-point Laplacian on an N^3 grid: diag 6, neighbours -1."""
    offs = _sorted_offsets(3, False)
    n, cols, vals, valid = _stencil((N, N, N), offs, lambda o: 6.0 if not any(o) else -1.0)
    return _assemble(n, cols, vals, valid, f"stencil3d_7pt_{N}")


def stencil3d_27pt(N: int) -> Csr:
    """3D 27-point stencil on an N^3 grid: diag 26, all 26 neighbours -1."""
    offs = _sorted_offsets(3, True)
    n, cols, vals, valid = _stencil((N, N, N), offs, lambda o: 26.0 if not any(o) else -1.0)
    return _assemble(n, cols, vals, valid, f"stencil3d_27pt_{N}")


def convdiff3d_7pt(N: int, peclet: float) -> Csr:
    """Upwind 3D convection-diffusion, velocity along +x,+y,+z with cell Peclet P.

    Row: diagonal 6 + 3P, upstream neighbours (offset -1 on an axis) -1 - P,
    downstream neighbours -1.  Dirichlet boundary by truncation.
    """
    P = float(peclet)
    offs = _sorted_offsets(3, False)

    def w(o):
        if not any(o):
            return 6.0 + 3.0 * P
        return (-1.0 - P) if min(o) < 0 else -1.0

    n, cols, vals, valid = _stencil((N, N, N), offs, w)
    return _assemble(n, cols, vals, valid, f"convdiff3d_7pt_{N}_P{P:g}")


def _varcoef(shape, coef: np.ndarray, name: str) -> Csr:
    """Variable-coefficient diffusion from per-cell coefficients (harmonic faces)."""
    dim = len(shape)
    offs = _sorted_offsets(dim, False)
    n, coords = _coords(shape)
    strides = [int(np.prod(shape[:a])) for a in range(dim)]
    lin = np.arange(n, dtype=np.int64)
    c = coef.reshape(-1).astype(np.float64)
    S = len(offs)
    cols = np.zeros((n, S), dtype=np.int32)
    vals = np.zeros((n, S), dtype=np.float64)
    valid = np.zeros((n, S), dtype=bool)
    diag = np.zeros(n, dtype=np.float64)
    centre = None
    for s, off in enumerate(offs):
        if not any(off):
            centre = s
            continue
        a = int(np.flatnonzero(off)[0])
        d = off[a]
        cc = coords[a] + d
        ok = (cc >= 0) & (cc < shape[a])
        nb = np.where(ok, lin + d * strides[a], lin)
        cn = c[nb]
        face = np.where(ok, 2.0 * c * cn / (c + cn), c)
        diag += face
        valid[:, s] = ok
        cols[:, s] = np.where(ok, nb, 0)
        vals[:, s] = -face
    valid[:, centre] = True
    cols[:, centre] = lin
    vals[:, centre] = diag
    return _assemble(n, cols, vals, valid, name)


def varcoef2d_5pt(N: int, rng: np.random.Generator) -> Csr:
    """2D 5-point variable-coefficient diffusion; draws N*N standard normals."""
    coef = np.exp(rng.standard_normal(N * N))
    return _varcoef((N, N), coef, f"varcoef2d_5pt_{N}")


def varcoef3d_7pt(N: int, rng: np.random.Generator) -> Csr:
    """3D 7-point variable-coefficient diffusion; draws N^3 standard normals."""
    coef = np.exp(rng.standard_normal(N * N * N))
    return _varcoef((N, N, N), coef, f"varcoef3d_7pt_{N}")


def powerlaw(n: int, seed: int = 0, lam: float | None = None, max_len: int = 10000) -> Csr:
    """Random power-law matrix.

    Draw order from ``default_rng(seed)``: Z = zipf(2.0, n); row lengths
    L = clip(Z, 1, max_len) (or clip(ceil(lam*Z), 1, max_len) when ``lam`` is
    given); then nnz uniform columns in [0, n) (row-major, unsorted, duplicates
    kept); then nnz standard-normal values.
    """
    rng = np.random.default_rng(seed)
    z = rng.zipf(2.0, n).astype(np.float64)
    if lam is not None:
        z = np.ceil(lam * z)
    lengths = np.clip(z, 1, max_len).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lengths, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = rng.integers(0, n, size=nnz, dtype=np.int64).astype(np.int32)
    val = rng.standard_normal(nnz)
    tag = "" if lam is None else f"_lam{lam:g}"
    return Csr(n, n, row_ptr.astype(np.int32), col, val, f"powerlaw_{n}{tag}")


def banded(n: int, half_bw: int = 64, fill: float = 0.3, seed: int = 0) -> Csr:
    """Random banded matrix.

    Draw order from ``default_rng(seed)``: for each row (row-major), 2*half_bw
    uniforms for the off-diagonal slots j = i-hb..i-1, i+1..i+hb (slots outside
    the matrix still consume a draw), a slot is present when its uniform is
    below ``fill``; the diagonal is always present; then one U[-1,1] value per
    present entry in row-major, ascending-column order.
    """
    rng = np.random.default_rng(seed)
    hb = half_bw
    offs = np.concatenate([np.arange(-hb, 0), np.arange(1, hb + 1)])
    present = np.empty((n, 2 * hb), dtype=bool)
    chunk = 65536
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        present[r0:r1] = rng.random((r1 - r0, 2 * hb)) < fill
    rows = np.arange(n, dtype=np.int64)[:, None]
    cols_all = rows + offs[None, :]
    present &= (cols_all >= 0) & (cols_all < n)
    # insert the diagonal between the lower and upper halves (ascending columns)
    valid = np.concatenate([present[:, :hb], np.ones((n, 1), bool), present[:, hb:]], axis=1)
    cols = np.concatenate([cols_all[:, :hb], rows, cols_all[:, hb:]], axis=1)
    cols = np.where(valid, cols, 0).astype(np.int32)
    del present, cols_all
    counts = valid.sum(axis=1, dtype=np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = np.ascontiguousarray(cols[valid])
    del cols, valid
    val = rng.uniform(-1.0, 1.0, size=col.size)
    return Csr(n, n, row_ptr.astype(np.int32), col, val, f"banded_{n}_hb{hb}")


def uniform_vector(n: int, rng: np.random.Generator) -> np.ndarray:
    """U[-1, 1] float64 vector of length n."""
    return rng.uniform(-1.0, 1.0, size=n)


def laplace2d_problem(N: int = 64, seed: int = 0):
    """2D 5-point Laplacian with x and b ~ U[-1,1] from default_rng(seed) (x first)."""
    A = laplace2d_5pt(N)
    rng = np.random.default_rng(seed)
    x = uniform_vector(A.n_rows, rng)
    b = uniform_vector(A.n_rows, rng)
    return A, x, b


def batch_sides(count: int = 4096, lo: int = 8, hi: int = 64, seed: int = 0) -> np.ndarray:
    """Grid sides rint(exp(U(ln lo, ln hi))) from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), count))).astype(np.int64)


def batch_system(i: int, side: int, seed: int = 0):
    """System i of the batched workload: varcoef 2D 5-point, b ~ U[-1,1].

    Uses ``default_rng([seed, i])``: side^2 standard normals for the cell
    coefficients, then side^2 uniforms for b.
    """
    rng = np.random.default_rng([seed, i])
    A = varcoef2d_5pt(int(side), rng)
    b = uniform_vector(A.n_rows, rng)
    return A, b


def random_csr(n_rows: int, n_cols: int, density: float, rng: np.random.Generator,
               integer_values: bool = False, empty_rows: float = 0.0, sort_cols: bool = True) -> Csr:
    """Small random CSR matrix for tests (optionally with integer values / empty rows)."""
    mask = rng.random((n_rows, n_cols)) < density
    if empty_rows > 0:
        mask[rng.random(n_rows) < empty_rows] = False
    lengths = mask.sum(axis=1)
    row_ptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(lengths, out=row_ptr[1:])
    cols = []
    for r in range(n_rows):
        c = np.flatnonzero(mask[r])
        if not sort_cols:
            c = rng.permutation(c)
        cols.append(c)
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    nnz = int(row_ptr[-1])
    if integer_values:
        val = rng.integers(-4, 5, size=nnz).astype(np.float64)
    else:
        val = rng.uniform(-1.0, 1.0, size=nnz)
    return Csr(n_rows, n_cols, row_ptr.astype(np.int32), col, val, "random")


def rows_csr(lengths, n_cols: int, rng: np.random.Generator) -> Csr:
    """CSR with the given row lengths, uniform random columns and U[-1,1] values."""
    lengths = np.asarray(lengths, dtype=np.int64)
    row_ptr = np.zeros(lengths.size + 1, dtype=np.int64)
    np.cumsum(lengths, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = rng.integers(0, n_cols, size=nnz).astype(np.int32)
    val = rng.uniform(-1.0, 1.0, size=nnz)
    return Csr(int(lengths.size), n_cols, row_ptr.astype(np.int32), col, val, "rows")
