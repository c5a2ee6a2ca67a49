/*
 * gko.h -- C ABI of the GB300-native sparse-solver hot path.
 *
 * The paper (Ginkgo's CUDA-to-HIP port, Section 1 contributions list) names
 * the sparse formats Coo, Csr, Ell and Hybrid and the Krylov solvers CG,
 * BiCG(STAB) and GMRES built on SpMV; Section 4 times SpMV kernels and
 * 1,000 CG iterations.  It prints no algorithm for any of them, so each entry
 * point below cites the section that names the operation and the textbook
 * definition it computes.
 *
 * Conventions shared by every entry point
 *   - Every call returns an int status (GKO_OK = 0, codes below).  No C++
 *     exception crosses this boundary and nothing aborts.  gko_last_error()
 *     returns a message for the calling thread's last failure.
 *   - Indices are int32 (nnz < 2^31); sizes are int64.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     stream-ordered.  Calls that report a host-side result (matrix creation,
 *     conversions, solves, gko_dot) synchronise that stream before returning.
 *   - Vectors (x, y, b) are caller-owned DEVICE pointers on the current
 *     device, contiguous, with the dtype given.  Matrix arrays passed to
 *     gko_matrix_create_csr are copied into library-owned device memory; the
 *     caller keeps its arrays.
 *   - A gko_matrix is immutable after creation; one handle may be used by
 *     several streams at once.  Every call that needs scratch memory takes it
 *     from a stream-ordered pool, so concurrent calls never share scratch.
 *   - The hot path runs only in this library's CUDA kernels (sm_103a).  There
 *     is no CPU fallback: without a usable GPU calls return GKO_CUDA_ERROR.
 */
#ifndef GKO_GB300_H
#define GKO_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define GKO_API __attribute__((visibility("default")))
#else
#define GKO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ statuses -- */
#define GKO_OK 0
#define GKO_INVALID_ARG 1        /* null pointer, bad sizes, malformed CSR      */
#define GKO_OUT_OF_MEMORY 2      /* device allocation failed                    */
#define GKO_FORMAT_UNSUITABLE 3  /* ELL padding above the configured limit      */
#define GKO_NOT_CONVERGED 4      /* iteration cap reached; x holds last iterate */
#define GKO_BREAKDOWN 5          /* exact-zero pivot in the Krylov recurrence   */
#define GKO_TIMEOUT 6            /* a bounded device wait gave up               */
#define GKO_CUDA_ERROR 7         /* a CUDA runtime call failed                  */
#define GKO_BUDGET_EXCEEDED 8    /* allocation would exceed the memory budget   */
#define GKO_NOT_SUPPORTED 9      /* dtype/format combination not provided       */

typedef struct gko_matrix_s *gko_matrix;

/* Value types.  GKO_F64 accumulates in FP64; GKO_F32 and GKO_BF16 values
 * accumulate in FP32 (vectors are FP32 for both). */
typedef enum { GKO_F64 = 0, GKO_F32 = 1, GKO_BF16 = 2 } gko_dtype;

/* Storage formats (paper, Section 1: Coo, Csr, Ell, Hybrid). */
typedef enum { GKO_CSR = 0, GKO_ELL = 1, GKO_COO = 2, GKO_HYBRID = 3, GKO_SELLP = 4 } gko_format;

/* Message for the calling thread's last non-OK status ("" if none). */
GKO_API const char *gko_last_error(void);
GKO_API const char *gko_status_string(int status);

/* Synchronise `stream` and report device-side failures recorded since the
 * last call: GKO_TIMEOUT when a bounded wait inside a kernel gave up (the
 * kernel then returned without finishing its work).  Clears the record. */
GKO_API int gko_device_status(void *stream);

/* Library version (major*10000 + minor*100 + patch). */
GKO_API int gko_version(void);

/* Limit on library-owned device memory in bytes (0 = unlimited, the
 * default).  Matrix storage and solver workspaces count against it; a call
 * that would exceed it returns GKO_BUDGET_EXCEEDED and allocates nothing.
 * Bytes currently held are returned through *in_use when it is non-NULL. */
GKO_API int gko_set_memory_budget(int64_t bytes);
GKO_API int gko_memory_in_use(int64_t *in_use);

/* ------------------------------------------------------------ matrices -- */

/* Create a CSR matrix (paper, Section 1: Csr) from row_ptr[n_rows+1],
 * col_idx[nnz] and values[nnz] of type `dtype`.  The arrays are host
 * pointers when values_on_device == 0, device pointers otherwise.  Column
 * order within a row is kept as given (unsorted allowed); duplicate (row,
 * col) entries are kept and summed by SpMV.
 * Checks (on the device): row_ptr[0] == 0, row_ptr[n_rows] == nnz,
 * row_ptr non-decreasing, 0 <= col < n_cols; any failure -> GKO_INVALID_ARG.
 * Also builds the load-balancing plan of the CSR SpMV: the row-length
 * histogram, the subwarp width for ordinary rows and the nonzero split of
 * long rows.  Synchronises `stream`.  *out receives the new handle. */
GKO_API int gko_matrix_create_csr(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t *row_ptr,
                          const int32_t *col_idx, const void *values, gko_dtype dtype,
                          int values_on_device, void *stream, gko_matrix *out);

/* Column-major ELL (paper, Section 1: Ell; layout of Bell & Garland, SC'09):
 * width K = longest row, stride = n_rows rounded up to 32, entry k of row i
 * at k*stride + i, padding col = -1 and value +0.0.  Returns
 * GKO_FORMAT_UNSUITABLE when K*n_rows > max_fill * nnz (max_fill <= 0 means
 * the default limit of 8).  Entries keep CSR storage order. */
GKO_API int gko_matrix_convert_to_ell(gko_matrix csr, double max_fill, void *stream, gko_matrix *out);

/* Row-major COO (paper, Section 1: Coo): the CSR entries in storage order
 * with an explicit int32 row index each. */
GKO_API int gko_matrix_convert_to_coo(gko_matrix csr, void *stream, gko_matrix *out);

/* Hybrid ELL + COO (paper, Section 1: Hybrid; Bell & Garland's HYB): the
 * first min(len_i, K) entries of each row in ELL of width K, the rest in a
 * row-major COO tail.  ell_width < 0 picks K as the largest k with
 * #{rows: len >= k} >= max(4096, n_rows/3); K = 0 gives a pure COO tail. */
GKO_API int gko_matrix_convert_to_hybrid(gko_matrix csr, int32_t ell_width, void *stream, gko_matrix *out);

/* SELL-P, sliced ELL with padding (paper, Section 1: Sellp, the format of its
 * Section 4 SpMV and CG measurements; layout of Anzt, Tomov & Dongarra 2014):
 * rows are cut into slices of `slice_size` consecutive rows (32, 64, 128 or
 * 256; <= 0 means 64), no reordering; slice s is as wide as its longest row
 * w_s and stores its entries column-major: entry k of row i (s = i /
 * slice_size) at (sets[s] + k) * slice_size + i % slice_size, sets[s] = w_0 +
 * ... + w_{s-1}.  Padding col = -1 and value +0.0; entries keep CSR storage
 * order.  Returns GKO_FORMAT_UNSUITABLE when the stored slots exceed
 * max_fill * nnz (max_fill <= 0 means the default limit of 8). */
GKO_API int gko_matrix_convert_to_sellp(gko_matrix csr, int32_t slice_size, double max_fill, void *stream,
                                        gko_matrix *out);

/* Copy of `m` (any format) with values converted to `to` (round to nearest
 * even); index arrays are shared with `m`, which must outlive the copy only
 * as far as the caller's own handle goes (sharing is reference counted). */
GKO_API int gko_matrix_convert_values(gko_matrix m, gko_dtype to, void *stream, gko_matrix *out);

/* Sizes and layout of a handle.  Any output pointer may be NULL.
 * ell_width / coo_nnz are 0 where the format has no such part; bytes is the
 * device memory owned (shared index arrays counted in full).  For SELL-P,
 * ell_width is the widest slice, ell_stride the slice size and coo_nnz the
 * number of stored slots (entries plus padding). */
GKO_API int gko_matrix_info(gko_matrix m, gko_format *format, gko_dtype *dtype, int64_t *n_rows,
                    int64_t *n_cols, int64_t *nnz, int32_t *ell_width, int64_t *ell_stride,
                    int64_t *coo_nnz, int64_t *bytes);

/* Copy the device arrays of `m` into caller HOST buffers (any may be NULL):
 *   CSR:    row_ptr[n_rows+1], col[nnz], val[nnz]
 *   ELL:    ell_col[K*stride], ell_val[K*stride]
 *   COO:    coo_row[nnz], coo_col[nnz], coo_val[nnz]
 *   HYBRID: ell_* for the ELL part and coo_* for the tail
 *   SELLP:  row_ptr[n_slices+1] receives the slice offsets sets[], ell_col /
 *           ell_val the stored slots (coo_nnz of gko_matrix_info of them)
 * Values are written in the handle's dtype.  Synchronises `stream`. */
GKO_API int gko_matrix_export(gko_matrix m, int32_t *row_ptr, int32_t *col, void *val, int32_t *ell_col,
                      void *ell_val, int32_t *coo_row, int32_t *coo_col, void *coo_val,
                      void *stream);

/* Load-balancing plan of a CSR or COO handle (CSR: built at creation from
 * the row-length histogram; COO: taken from the CSR it was converted from).
 * CSR kernel 1, the row-block kernel (regular matrices: longest row <= 4x
 * the mean): row blocks stream into shared memory by bulk copies in stages
 * of stage_cap entries; `subwarp` lanes sum each row, each subwarp owning
 * rows_per_subwarp interleaved rows of a block of 128 threads.
 * Handles with FP32 or BF16 values use a quarter of the FP64 lanes per row
 * (at least 1) and, when that changes the width, two rows per subwarp.
 * CSR kernel 2, the merge-path kernel: the merged sequence of row ends and
 * nonzeros is split into equal shares per thread, so long rows spread over
 * many threads and tiles.
 * CSR kernel 3, the nonzero split (skewed matrices, the default there): the
 * nonzeros are cut into equal tiles of
 * 1024, 8 consecutive ones per thread; each tile finds its rows in a staged
 * slice of row_ptr (one row index per tile is precomputed), and rows that
 * cross threads or tiles are completed from carries in a fixed order.
 * CSR kernel 0, the subwarp kernel: `subwarp` lanes per row,
 * rows_per_subwarp rows per pass, and rows longer than long_threshold split
 * into fixed-size nonzero chunks (n_long_rows rows, n_long_chunks chunks).
 * COO kernel 1: the row-block schedule over the COO arrays (row blocks start
 * at precomputed entries; each stage also carries the row indices, from
 * which the block finds its rows' ranges); COO kernel 0: the tiled segmented
 * reduction (the paper's COO scheme, the default for skewed matrices).
 * hist33: row-length histogram in log2 classes (hist[0]: empty rows;
 * hist[b], b >= 1: lengths in [2^(b-1), 2^b)).  Any output may be NULL.
 * GKO_INVALID_ARG for other formats. */
GKO_API int gko_matrix_plan(gko_matrix m, int32_t *kernel, int32_t *subwarp, int32_t *rows_per_subwarp,
                            int32_t *stage_cap, int32_t *long_threshold, int64_t *n_long_rows,
                            int64_t *n_long_chunks, int64_t *hist33);

/* Override the plan (the autotuner's knob).  CSR kernel 0: subwarp S in
 * 1,2,4,8,16,32, R in 1,2,4, long-row threshold 32*S; CSR kernel 1:
 * row-block, S in 1,2,4,8, R in 1,2,4, stage_cap a power of two in
 * 512..8192 (ignored otherwise); CSR kernel 2: merge path, kernel 3: nonzero
 * split (S, R still validated, unused).  COO kernel 1: row-block, S in 1,2,4,8, R in 1,2,4,
 * stage_cap a power of two in 512..4096; COO kernel 0 or 2: segmented
 * reduction.  The solvers' cached low-precision copies follow; handles made by
 * gko_matrix_convert_values keep their own plan.  Synchronises `stream`. */
GKO_API int gko_matrix_set_plan(gko_matrix m, int32_t kernel, int32_t subwarp, int32_t rows_per_subwarp,
                                int32_t stage_cap, void *stream);

/* SpMV plan autotuner (the project's tuner for lanes per row, rows per
 * subwarp, stage capacity and kernel; the paper tunes nothing at run time):
 * for a CSR handle it times every row-block plan (subwarp 1,2,4,8 x rows per
 * subwarp 1,2,4 x stage_cap 512,1024,2048), the merge path, the nonzero split
 * and the subwarp kernel with subwarp 4..32; for a COO handle the row-block plans and the
 * segmented reduction.  keep_kernel != 0 keeps the handle's kernel and tunes
 * only its parameters (row-block plans; nothing to tune for the nonzero
 * split, the merge path and the segmented reduction), so the kernel choice
 * stays the histogram rule's whatever the timing conditions.  Each candidate runs y = A x once
 * untimed, then `reps` times (1..100) with L2 flushed (256 MB write) before
 * each, best time kept; the three fastest are timed again the same way with
 * 3*reps runs, and the fastest of those is set on the handle (as
 * gko_matrix_set_plan) and
 * returned (outputs may be NULL; best_ms in milliseconds).  x, y: device
 * vectors of the SpMV's vector dtype; y is overwritten.  Synchronises
 * `stream`.  GKO_NOT_SUPPORTED for other formats. */
GKO_API int gko_matrix_tune(gko_matrix m, const void *x, void *y, int32_t reps, int32_t keep_kernel,
                            int32_t *kernel, int32_t *subwarp, int32_t *rows_per_subwarp, int32_t *stage_cap,
                            float *best_ms, void *stream);

GKO_API int gko_matrix_destroy(gko_matrix m);

/* ----------------------------------------------------------------- SpMV -- */

/* y = alpha * A * x + beta * y  (paper, Section 4: the SpMV kernels timed).
 * alpha, beta: HOST scalars.  x[n_cols], y[n_rows]: device vectors of
 * `vec_dtype`, which must be GKO_F64 for an F64 matrix and GKO_F32 for F32
 * and BF16 matrices.  beta == 0 overwrites y without reading it (NaN in y
 * does not propagate); NaN/Inf in x propagate through every row that
 * references them, also when alpha == 0.  ELL padding never reads x.
 * Deterministic: the same inputs give bit-identical y on every call.
 * x and y must not overlap.  Asynchronous on `stream`. */
GKO_API int gko_spmv(const double *alpha, gko_matrix A, const void *x, const double *beta, void *y,
             gko_dtype vec_dtype, void *stream);

/* gko_spmv on HOST vectors: copies x_host (n_cols elements of vec_dtype) to
 * the caller's device buffer x_dev, and y_host to y_dev when beta != 0,
 * runs gko_spmv, and copies y_dev back to y_host, all in stream order on
 * `stream` (returns once enqueued; host buffers must stay valid until the
 * stream reaches the last copy, and should be page-locked for the copies to
 * be asynchronous).  Calls on different streams overlap one call's copies
 * with another's SpMV.  Errors as gko_spmv; null host or device buffers ->
 * GKO_INVALID_ARG. */
GKO_API int gko_spmv_host(const double *alpha, gko_matrix A, const void *x_host, const double *beta,
                          void *y_host, gko_dtype vec_dtype, void *x_dev, void *y_dev, void *stream);

/* y = alpha * A * x + beta * y for an F64 COO handle, allocating nothing.
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory at the time they multiply (their memory is owned by
 * another allocator, or an allocation's possible implicit synchronisation is
 * not acceptable in their loop).  It always runs the tiled segmented-reduction
 * kernels, whatever plan the handle carries, so its y equals gko_spmv's
 * within the SpMV tolerance (bit-identical under the default plan; a handle
 * set to the row-block COO plan sums in another order).  The per-tile
 * carries live in a fixed 2 MiB device array inside the library instead of
 * pool scratch.  At most 134,217,728 COO entries; larger handles are
 * rejected with GKO_INVALID_ARG.  CUDA loads this entry point's device code,
 * and with it the array, lazily: the first call on a device (which also
 * looks up the array's device address with cudaGetSymbolAddress, that
 * device current) allocates that module's memory once and may synchronise,
 * so make the first call on each device during set-up, before any stream
 * capture; from then on the array stays on that device until the process
 * exits and calls touch no allocator.  Every call shares the one array:
 * calls that overlap on the GPU (other streams, or other threads) race and
 * give wrong results; serialise them.  Asynchronous on `stream`. */
GKO_API int gko_spmv_coo_noalloc(const double *alpha, gko_matrix A, const double *x, const double *beta,
                                 double *y, void *stream);

/* ---------------------------------------------------------------- BLAS-1 -- */

/* Deterministic FP64 reductions and updates on device vectors of length n
 * (the vector kernels inside the Krylov solvers).  *result is a HOST double;
 * these calls synchronise `stream`. */
GKO_API int gko_dot(int64_t n, const double *x, const double *y, double *result, void *stream);
GKO_API int gko_nrm2(int64_t n, const double *x, double *result, void *stream);
/* y = a*x + y; asynchronous. */
GKO_API int gko_axpy(int64_t n, double a, const double *x, double *y, void *stream);
/* Fused multi-axpy + norm: y -= sum_j h[j] * V[j*ldv : j*ldv + n] for
 * j < k, then *result = ||y||_2 (host, synchronises).  h: host array. */
GKO_API int gko_multi_axpy_norm(int64_t n, int32_t k, const double *h, const double *V, int64_t ldv,
                        double *y, double *result, void *stream);
/* Fused multi-dot: h[j] = V[j] . w for j < k (h: host array; synchronises). */
GKO_API int gko_multi_dot(int64_t n, int32_t k, const double *V, int64_t ldv, const double *w,
                  double *h, void *stream);
/* Fused SpMV + dot: y = A x and *result = x . y (FP64, host; synchronises).
 * A must be square with FP64 values. */
GKO_API int gko_spmv_dot(gko_matrix A, const double *x, double *y, double *result, void *stream);

/* --------------------------------------------------------------- solvers -- */

#define GKO_PRECISION_F64 0        /* all FP64                                   */
#define GKO_PRECISION_MIXED_F32 1  /* FP32 inner solve + FP64 refinement         */
#define GKO_PRECISION_MIXED_BF16 2 /* BF16-valued inner SpMV + FP64 refinement   */

/* How mixed precision recovers FP64 accuracy (opts->refinement).
 * RESTART: iterative refinement; each step forms r = b - A x in FP64 and
 *      solves A d = r from scratch with FP32 (or BF16-valued) A, FP32 vectors,
 *      FP64 dots and scalars, then x += d in FP64 (Buttari et al. 2007).
 * RELIABLE (CG, BiCGSTAB): one run of the Krylov recurrences on the FP32 copy
 *      with FP32 vectors, FP64 dots and scalars, accumulating the iterate's
 *      change d in FP32; whenever the recurrence residual meets rel_tol ||b||
 *      or drops below reliable_delta times its largest norm since the last
 *      update, d is added to the FP64 x, r is replaced by the FP64 residual
 *      b - A x and the recurrences continue with their directions and
 *      scalars (reliable updates: Sleijpen & van der Vorst, Computing 56,
 *      1996; residual replacement without restart: van der Vorst & Ye, SIAM
 *      J. Sci. Comput. 22, 2000).  BiCGSTAB restarts only after a half step
 *      (||s|| small).  The solve converges when the replaced FP64 residual
 *      meets rel_tol ||b||; outer_iterations counts the updates; inner_tol,
 *      max_outer and inner_maxit are not used.  GMRES: GKO_NOT_SUPPORTED.
 * AUTO (0): RELIABLE for BiCGSTAB and for CG with more than 2^18 rows;
 *      RESTART for GMRES and for smaller CG systems (whose inner solves run
 *      as one single-launch CG each).
 * The FP32 (or BF16) copy of a CSR matrix with more than 2^18 rows whose
 * rows are nearly equal in length (ELL padding at most 1.2 x nnz) is stored
 * in ELL, which streams 4-byte values faster than the CSR kernels. */
#define GKO_REFINE_AUTO 0
#define GKO_REFINE_RESTART 1
#define GKO_REFINE_RELIABLE 2

/* Preconditioners (paper, Section 1 lists them beside the solvers; M =
 * diag(A), Saad, Iterative Methods for Sparse Linear Systems, Sec. 10.2).
 * JACOBI: CG becomes preconditioned CG (Saad Alg. 9.1) and BiCGSTAB is
 * right preconditioned; convergence is still judged on the unpreconditioned
 * residual ||b - A x||.  The inverse diagonal is built per solve from the FP64
 * matrix (diagonal duplicates summed, a zero diagonal taken as 1) and, for
 * mixed precision, rounded to FP32 for the inner solve.  GMRES with a
 * preconditioner returns GKO_NOT_SUPPORTED.
 * BLOCK_JACOBI: M = the diagonal blocks of A (Saad Sec. 12.2), blocks of
 * opts->block_size consecutive rows (the last one n % block_size rows when
 * the size does not divide n), each inverted once per solve by Gauss-Jordan
 * elimination with partial pivoting (as gko_block_jacobi_inverse); CG and
 * BiCGSTAB use it as JACOBI uses diag(A); mixed-precision recurrences apply
 * the inverse blocks rounded to FP32.  A CSR matrix only (otherwise
 * GKO_NOT_SUPPORTED); a block whose elimination meets an all-zero pivot
 * column leaves its rows unscaled, as a zero diagonal does for JACOBI.
 * Extra device memory: n * block_size doubles (and as many floats for
 * mixed precision). */
#define GKO_PRECOND_NONE 0
#define GKO_PRECOND_JACOBI 1
#define GKO_PRECOND_BLOCK_JACOBI 2

typedef struct {
  int32_t restart;      /* GMRES restart length m (<= 0: 30; at most 128)        */
  int32_t precision;    /* GKO_PRECISION_*                                       */
  double inner_tol;     /* mixed: inner relative tolerance (<= 0: 1e-5)          */
  int32_t max_outer;    /* mixed: refinement steps (<= 0: 30; GMRES: the larger of
                           30 and ceil(max_iters / (4 restart)))                */
  int32_t inner_maxit;  /* mixed: inner iteration cap per step (<= 0: max_iters;
                           GMRES: 4 restart cycles per step)                    */
  int32_t check_every;  /* host status poll interval in iterations (<= 0: auto)  */
  int32_t preconditioner; /* GKO_PRECOND_* (CG, BiCGSTAB)                        */
  int32_t refinement;   /* mixed: GKO_REFINE_* (0: AUTO)                         */
  int32_t block_size;   /* BLOCK_JACOBI: rows per diagonal block, 1..32 (<= 0: 8) */
  double reliable_delta; /* RELIABLE: update factor in [0, 1) (0: 0.1)            */
} gko_solve_opts;

typedef struct {
  int32_t status;           /* GKO_OK, GKO_NOT_CONVERGED or GKO_BREAKDOWN          */
  int32_t iterations;       /* Krylov iterations (inner ones for mixed precision) */
  int32_t outer_iterations; /* GMRES restart cycles / refinement steps            */
  int32_t reserved;
  double rel_residual;      /* true ||b - A x||_2 / ||b||_2, computed in FP64      */
} gko_solve_result;

/* Solve A x = b with Krylov methods (paper, Section 1:
 * CG, BiCG(STAB), GMRES; Section 4: CG timed on GPUs).
 *   A: square FP64 matrix of any format (for mixed precision an FP32 or
 *      BF16 copy is made once and cached on the handle);
 *   b[n], x[n]: device FP64 vectors; x holds x0 on entry, the solution on
 *      exit (also on NOT_CONVERGED / BREAKDOWN: the last iterate);
 *   stop when ||r_k|| <= rel_tol * ||b|| for the recurrence residual, then
 *      verify with the true residual b - A x; if the true residual misses,
 *      it replaces r and iteration goes on until max_iters;
 *   b == 0 gives x = 0 after 0 iterations.
 * CG: Hestenes-Stiefel (Saad Alg. 6.18); breakdown when p.Ap <= 0.
 * BiCGSTAB: van der Vorst 1992 (Saad Alg. 7.7); breakdown on exact zeros
 *      of rhat.r, rhat.v, t.t or omega.
 * GMRES(m): Saad-Schultz restarted GMRES with classical Gram-Schmidt and
 *      selective reorthogonalisation (a second pass when the first shrinks
 *      ||w|| below 1/sqrt(2) of its norm after A v_j) and Givens rotations on
 *      the device; iterations count
 *      Arnoldi steps, outer_iterations restart cycles; each cycle starts
 *      from the true residual.
 * Mixed precision (opts->precision): x stays FP64 and the method runs on an
 *      FP32 (or BF16-valued) copy of A with FP32 vectors, FP64 dots and FP64
 *      scalars, refined as opts->refinement says (GKO_REFINE_*).  RESTART:
 *      each refinement step forms r = b - A x in FP64, solves A d = r to
 *      ||r_inner|| <= inner_tol ||r|| and adds d in FP64, until
 *      ||b - A x|| <= rel_tol ||b|| or max_outer steps.  Bad refinement or
 *      reliable_delta: GKO_INVALID_ARG.
 * All scalars and convergence checks stay on the device; the host polls a
 * status word every few iterations.  *res is written before returning
 * (synchronises `stream`); opts may be NULL.  Returns res->status (GKO_OK,
 * GKO_NOT_CONVERGED, GKO_BREAKDOWN) or an error. */
GKO_API int gko_solve_cg(gko_matrix A, const double *b, double *x, double rel_tol, int32_t max_iters,
                 const gko_solve_opts *opts, gko_solve_result *res, void *stream);
GKO_API int gko_solve_bicgstab(gko_matrix A, const double *b, double *x, double rel_tol,
                       int32_t max_iters, const gko_solve_opts *opts, gko_solve_result *res,
                       void *stream);
GKO_API int gko_solve_gmres(gko_matrix A, const double *b, double *x, double rel_tol, int32_t max_iters,
                    const gko_solve_opts *opts, gko_solve_result *res, void *stream);

/* Block-Jacobi setup (the preconditioner of GKO_PRECOND_BLOCK_JACOBI; Saad,
 * Iterative Methods for Sparse Linear Systems, Sec. 12.2; Golub & Van Loan,
 * Matrix Computations, Sec. 3.4 for the elimination).  A: square FP64 CSR
 * matrix.  The diagonal blocks are rows and columns k*block_size ..
 * k*block_size + nb - 1, nb = min(block_size, n - k*block_size); each is
 * gathered densely (entries of a row summed in storage order) and inverted
 * by Gauss-Jordan elimination on [D | I] with partial pivoting (pivot: the
 * first row of largest magnitude in the column; the pivot row multiplied by
 * the reciprocal of the pivot; every other row r becomes row_r - m_r row_k,
 * each product and difference rounded separately).  B: device array of n * block_size
 * doubles, written with row i of its block's inverse at B[i*block_size ..
 * i*block_size + nb - 1] and zeros after it.  A block whose pivot column is
 * all zero at some step gets identity rows; *singular (host, nullable)
 * receives how many.  block_size: 1..32 (GKO_INVALID_ARG otherwise); other
 * formats or value types: GKO_NOT_SUPPORTED.  Synchronises `stream` when
 * singular is given. */
GKO_API int gko_block_jacobi_inverse(gko_matrix A, int32_t block_size, double *B, int64_t *singular,
                                     void *stream);

/* ------------------------------------------------------------ batched CG -- */

/* Many independent small SPD systems solved by CG in one persistent launch
 * (the CG of the paper's Section 1 solver list, per system).  Systems are
 * concatenated: system i has rows [row_off[i], row_off[i+1]) and nonzeros
 * [nnz_off[i], nnz_off[i+1]); its local row pointers (n_i + 1 entries, from
 * 0 to nnz_i) start at row_ptr[row_off[i] + i]; col holds local column
 * indices (0 <= col < n_i).  All arrays are HOST arrays, copied and checked
 * at creation (bad input -> GKO_INVALID_ARG); values are always FP64.
 * `storage` GKO_F64 keeps them; GKO_F32 rounds them to nearest FP32 on the
 * device (the same rounding as gko_matrix_convert_values), and the batch
 * then solves the FP32-rounded systems with FP64 arithmetic and vectors.
 * Systems may have up to 8192 rows.  Synchronises `stream`. */
typedef struct gko_batch_s *gko_batch;
GKO_API int gko_batch_create(int32_t count, const int64_t *row_off, const int64_t *nnz_off,
                             const int32_t *row_ptr, const int32_t *col, const double *values,
                             gko_dtype storage, void *stream, gko_batch *out);

/* The same from one CSR per system: system i has n_rows[i] rows, HOST arrays
 * row_ptrs[i] (n_rows[i] + 1 entries from 0), cols[i] and values[i] (FP64,
 * row_ptrs[i][n_rows[i]] entries each).  The library concatenates them and
 * builds the offsets; checks, storage and rounding as gko_batch_create. */
GKO_API int gko_batch_create_systems(int32_t count, const int32_t *n_rows, const int32_t *const *row_ptrs,
                                     const int32_t *const *cols, const double *const *values, gko_dtype storage,
                                     void *stream, gko_batch *out);

/* Copy the stored batch to HOST arrays in gko_batch_create's layout (any
 * pointer may be NULL to skip that array): row_off and nnz_off (count + 1),
 * row_ptr (total_rows + count), col (total_nnz) and values (total_nnz
 * elements of the storage type: double for F64, float for F32).
 * Synchronises `stream`. */
GKO_API int gko_batch_export(gko_batch B, int64_t *row_off, int64_t *nnz_off, int32_t *row_ptr, int32_t *col,
                             void *values, void *stream);

/* Solve every system: b, x are DEVICE FP64 vectors laid out like the rows
 * (x: x0 in, solution out).  Per system: stop when ||r_k|| <= rel_tol ||b_i||
 * and the true residual confirms (else it replaces r), or after max_iters.
 * The batch's schedule decides how: systems with at most warp_rows rows are
 * solved by one warp each, larger ones by a block of `threads` threads, from
 * the CSR arrays or from the batch's per-system ELL copy (both sum every row
 * in storage order, so the results are identical).  The launch is captured
 * once into a CUDA graph per (b, x, rel_tol, max_iters, stream, schedule) and
 * replayed.  iterations / rel_residuals (true residuals) / statuses: optional
 * HOST arrays of `count` entries.  Returns GKO_OK when every system
 * converged, else GKO_BREAKDOWN or GKO_NOT_CONVERGED.  Synchronises
 * `stream`. */
GKO_API int gko_batch_cg(gko_batch B, const double *b, double *x, double rel_tol, int32_t max_iters,
                         int32_t *iterations, double *rel_residuals, int32_t *statuses, void *stream);

#define GKO_BATCH_CSR 0 /* the concatenated CSR arrays                       */
#define GKO_BATCH_ELL 1 /* per-system column-major ELL (longest row's slots) */

/* Autotuner (the project's; the paper tunes nothing at run time): times the
 * whole batch for every schedule, warp_rows in {0, 64, 144, 256} x threads
 * per block in {256, 512, 1024} x storage CSR or ELL (solving from a scratch
 * copy of x0; x0 is not changed), keeps the fastest and reports it (outputs
 * may be NULL; best_ms in milliseconds).  Synchronises `stream`. */
GKO_API int gko_batch_tune(gko_batch B, const double *b, const double *x0, double rel_tol, int32_t max_iters,
                           int32_t *warp_rows, int32_t *threads, int32_t *storage, float *best_ms, void *stream);

/* Set the schedule directly: warp_rows >= 0 (0 = block mode only; capped at
 * 256), threads 256, 512 or 1024, storage GKO_BATCH_CSR or GKO_BATCH_ELL;
 * anything else -> GKO_INVALID_ARG.  gko_batch_set_threshold changes
 * warp_rows only.  The default: 144 rows, 256 threads, CSR. */
GKO_API int gko_batch_set_schedule(gko_batch B, int32_t warp_rows, int32_t threads, int32_t storage, void *stream);
GKO_API int gko_batch_set_threshold(gko_batch B, int32_t warp_rows, void *stream);

/* Precision of gko_batch_cg (and of gko_batch_tune's timings).
 * GKO_PRECISION_F64 (the default): FP64 vectors and arithmetic on the stored
 * values.  GKO_PRECISION_MIXED_F32: per system, CG with reliable updates
 * (Sleijpen & van der Vorst, Computing 56, 1996; residual replacement
 * without restart, van der Vorst & Ye, SIAM J. Sci. Comput. 22, 2000): the
 * recurrences run on the FP32 rounding of the stored values with FP32
 * vectors (r, p, q and the iterate's change), FP64 dots and FP64 scalars;
 * when the recurrence residual meets rel_tol ||b_i|| or drops below
 * reliable_delta (0: 0.1) times its largest norm since the last update, the
 * change is added to the FP64 x and r is replaced by b - A x computed in FP64
 * with the stored values; a system converges when that FP64 residual meets
 * rel_tol ||b_i||.  The FP32 values are made once (FP64 storage) or are the
 * stored ones (FP32 storage).  Bad arguments: GKO_INVALID_ARG.  Synchronises
 * `stream`. */
GKO_API int gko_batch_set_precision(gko_batch B, int32_t precision, double reliable_delta, void *stream);

/* Reliable updates per system (`count` HOST entries) of the last
 * gko_batch_cg call: zeros after an FP64 solve.  Synchronises `stream`. */
GKO_API int gko_batch_last_updates(gko_batch B, int32_t *updates, void *stream);

/* The batch's sizes and schedule (outputs may be NULL). */
GKO_API int gko_batch_info(gko_batch B, int32_t *count, int64_t *total_rows, int64_t *total_nnz,
                           int32_t *warp_rows, int32_t *n_items, int32_t *threads, int32_t *storage);
GKO_API int gko_batch_destroy(gko_batch B);

/* --------------------------------------------------------------- serving -- */

/* Request loop with continuous batching over resident matrices.  `slots`
 * worker threads, each with its own CUDA stream on the current device, take
 * the oldest queued request as soon as a slot is free and its device-memory
 * estimate (b, x, solver workspace and preconditioner) fits in budget_bytes together with
 * the resident matrices and the requests already running (budget_bytes = 0:
 * no limit).  Solves of different requests overlap on the GPU; each result
 * is the one the same call gives alone (deterministic kernels).  Mixed-
 * precision requests create the matrix's low-precision copy on first use. */
typedef struct gko_server_s *gko_server;
GKO_API int gko_server_create(int32_t slots, int64_t budget_bytes, gko_server *out);

/* Register a resident square F64 matrix (the caller keeps the handle alive
 * until the server is destroyed).  GKO_BUDGET_EXCEEDED if the resident set
 * would exceed the budget. */
GKO_API int gko_server_add_matrix(gko_server S, gko_matrix A, int32_t *matrix_id);

/* Queue a solve of A_matrix_id x = b (b: HOST array of n doubles, copied at
 * submission; x0 = 0) with solver 0 CG, 1 BiCGSTAB, 2 GMRES.  Returns at
 * once with *request_id.  GKO_BUDGET_EXCEEDED if the request alone cannot
 * fit the budget; GKO_INVALID_ARG for an unknown matrix or bad arguments. */
GKO_API int gko_server_submit(gko_server S, int32_t matrix_id, int32_t solver, const double *b, double rel_tol,
                              int32_t max_iters, const gko_solve_opts *opts, int64_t *request_id);

/* Result of a request: wait != 0 blocks until it is done.  *done = 0 while
 * it runs (non-blocking call).  When done: *res, the solution in x (HOST, n
 * doubles; may be NULL) and the submission-to-result latency in ms (may be
 * NULL); the request is then forgotten.  Returns the solve's status. */
GKO_API int gko_server_result(gko_server S, int64_t request_id, int wait, int32_t *done,
                              gko_solve_result *res, double *x, double *latency_ms);

/* Completed requests, latency percentiles (ms, submission to result) and
 * completions per second between the first submission and the last
 * completion; peak number of solves running at once. */
GKO_API int gko_server_stats(gko_server S, int64_t *completed, double *p50_ms, double *p99_ms,
                             double *solves_per_s, int32_t *peak_active);

/* Stop the workers (requests still queued are dropped) and free the server. */
GKO_API int gko_server_destroy(gko_server S);

/* --------------------------------------------------- diagnostics -- */

/* Subwarp reduction microbenchmark (paper, Section 3.3: the reduce listing
 * and its inner-loop difference method).  data: `n` device values of
 * `dtype` (F64 or F32), n a positive multiple of 256; each value is one
 * thread's input and receives its output.  Every thread runs `inner_loops`
 * butterfly reductions over subwarps of `subwarp` consecutive lanes (1, 2,
 * 4, 8, 16 or 32): in each of log2(subwarp) steps a lane adds the value of
 * the lane whose index differs in one bit.  impl 0: the library's subwarp
 * primitive; 1: CUDA cooperative groups tiled_partition; 2: the full-warp
 * xor shuffle.  Stream-ordered; time two calls (e.g. 2000 and 1000 loops)
 * and subtract.  GKO_INVALID_ARG on bad sizes. */
GKO_API int gko_bench_subwarp_reduce(int32_t subwarp, int32_t impl, gko_dtype dtype, int32_t inner_loops,
                                     void *data, int64_t n, void *stream);

/* FMA throughput probe (no counterpart in the paper; it measures the FP64
 * pipe that co-limits the FP64 kernels on this GPU).  data: `n` device values
 * of `dtype` (F64 or F32), n a positive multiple of 256; each is one
 * thread's seed.  Every thread runs 8 independent chains v = fma(v, a, b)
 * (a = 1 - 2^-10, b = 2^-10; chain c starts at seed + c/8) for `inner_loops`
 * steps in registers and overwrites its value with the sum of its chains.
 * n * 8 * inner_loops FMAs per call; time two loop counts and subtract.
 * Stream-ordered.  GKO_INVALID_ARG on bad sizes or dtype. */
GKO_API int gko_bench_fma(gko_dtype dtype, int32_t inner_loops, void *data, int64_t n, void *stream);

/* Random-gather throughput probe (no counterpart in the paper; it measures
 * the access pattern that bounds SpMV on matrices with uniformly random
 * columns: one element per L2 sector).  x: 2^log2_len device elements of
 * `dtype` (F64: 8 bytes, F32: 4 bytes; log2_len 1..30), read as raw bits;
 * out: `n` elements (n a positive multiple of 256, n * 8 < 2^32), one per
 * thread.  Thread t keeps 8 streams with states s_c = 8 t + c; each of
 * `inner_loops` steps sets s_c = 1664525 s_c + 1013904223 (mod 2^32) and
 * xors element (s_c >> (32 - log2_len)) of x into its accumulator (loaded
 * bypassing L1), which it writes to out[t].  n * 8 * inner_loops gathers
 * per call; time two loop counts and subtract.  Stream-ordered.
 * GKO_INVALID_ARG on bad sizes or dtype. */
GKO_API int gko_bench_gather(gko_dtype dtype, int32_t inner_loops, const void *x, int32_t log2_len, void *out,
                             int64_t n, void *stream);

/* Failure-detection check (no counterpart in the paper): one warp waits on a
 * shared-memory barrier that nothing completes, through the bounded wait the
 * bulk-copy SpMV kernels use, for at most `cycles` clock cycles (1 .. 2^32).
 * The wait gives up, the kernel records GKO_TIMEOUT in the device error word
 * (read and cleared by gko_device_status) and returns; *timed_out = 1.
 * Synchronises `stream`; the context stays usable. */
GKO_API int gko_diag_bounded_wait(int64_t cycles, int32_t *timed_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GKO_GB300_H */
