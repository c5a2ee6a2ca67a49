/*
 * Plain CPU oracle for the sparse hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  The product path never calls it.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * Everything here is the plain definition, computed sequentially in IEEE
 * double (compiled with -ffp-contract=off, so no fused multiply-adds):
 *
 *   SpMV      y = alpha*A*x + beta*y  for the formats the paper lists
 *             (Coo, Csr, Ell, Hybrid, Sellp; Section 1, contributions list).
 *             Each row sum runs left to right in storage order.  beta == 0
 *             overwrites y without reading it (BLAS convention).
 *   Formats   ELL / COO / HYB as defined by Bell & Garland, "Implementing
 *             sparse matrix-vector multiplication on throughput-oriented
 *             processors", SC'09.  ELL is column-major with stride
 *             round_up(n, 32), padding col = -1, val = +0.0.
 *   Solvers   CG (Hestenes & Stiefel 1952; Saad, Iterative Methods for Sparse
 *             Linear Systems, 2nd ed., Alg. 6.18), BiCGSTAB (van der Vorst
 *             1992; Saad Alg. 7.7), restarted GMRES(m) with modified
 *             Gram-Schmidt and Givens rotations (Saad & Schultz 1986; Saad
 *             Alg. 6.9/6.11), and mixed-precision iterative refinement (an
 *             FP64 outer residual loop around an inner solve whose matrix and
 *             vectors are stored in FP32; Buttari et al. 2007).
 *   Precond.  Jacobi M = diag(A) (Saad Sec. 10.2) and block-Jacobi M = the
 *             diagonal blocks of A, inverted by Gauss-Jordan elimination with
 *             partial pivoting (Saad Sec. 12.2; Golub & Van Loan, Matrix
 *             Computations, Sec. 3.4).
 *
 * The paper (Section 1) names these formats and solvers but prints no
 * algorithm for them, so the textbook definitions above are the reference.
 * Readings taken where the paper is silent:
 *   - stopping: ||r_k|| <= tol*||b|| on the recurrence residual, then the true
 *     residual b - A x is formed; if that misses the tolerance it replaces r
 *     and the iteration goes on (CG keeps p; BiCGSTAB restarts its
 *     recurrences); the reported residual is always the true one;
 *   - b == 0 returns x = 0 after 0 iterations;
 *   - breakdown on exact zeros only: CG p.q <= 0; BiCGSTAB rhat.r == 0,
 *     rhat.v == 0, t.t == 0 or omega == 0; GMRES a zero rotation denominator.
 *     GMRES h_{j+1,j} == 0 is a lucky breakdown (exact solve).
 *   - hybrid ELL width K = largest k with #{rows: len >= k} >= 4096 and
 *     3 * #{rows: len >= k} >= n (Bell-Garland heuristic); K = 0 is pure COO.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_OK = 0, OR_NOT_CONVERGED = 4, OR_BREAKDOWN = 5, OR_INVALID = 1 };

static int g_threads = 1;

/* Threads used by the row-parallel SpMV loops (CSR and ELL only; each row is
 * still summed sequentially so the result does not depend on the count). */
int or_set_threads(int t) {
#ifdef _OPENMP
  g_threads = t > 0 ? t : omp_get_max_threads();
  return g_threads;
#else
  (void)t;
  g_threads = 1;
  return 1;
#endif
}

int or_has_openmp(void) {
#ifdef _OPENMP
  return 1;
#else
  return 0;
#endif
}

/* ---------------------------------------------------------------- SpMV -- */

void or_spmv_csr(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                 const double *x, double alpha, double beta, double *y) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4096) num_threads(g_threads)
#endif
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += val[k] * x[col[k]];
    y[i] = beta == 0.0 ? alpha * s : alpha * s + beta * y[i];
  }
}

/* FP32 values, FP32 x and y, FP32 accumulation: every product and every
 * partial sum is rounded to float. */
void or_spmv_csr_f32(int64_t n, const int32_t *rp, const int32_t *col, const float *val,
                     const float *x, float alpha, float beta, float *y) {
  for (int64_t i = 0; i < n; ++i) {
    float s = 0.0f;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      float p = val[k] * x[col[k]];
      s = s + p;
    }
    y[i] = beta == 0.0f ? alpha * s : alpha * s + beta * y[i];
  }
}

/* Error-free transformations (Dekker/Knuth TwoSum, FMA-based TwoProduct)
 * with Neumaier accumulation: a near-exact row sum used to attribute a
 * parity failure to summation order.  fma() is the correctly rounded C99
 * function, so p + e == a*b exactly. */
void or_spmv_csr_exact(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                       const double *x, double alpha, double beta, double *y) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0, c = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      double a = val[k], b = x[col[k]];
      double p = a * b;
      double e = fma(a, b, -p);
      double t = s + p;
      c += (fabs(s) >= fabs(p)) ? (s - t) + p : (p - t) + s;
      s = t;
      c += e;
    }
    double row = s + c;
    y[i] = beta == 0.0 ? alpha * row : alpha * row + beta * y[i];
  }
}

int64_t or_ell_stride(int64_t n) { return (n + 31) / 32 * 32; }

int32_t or_ell_width(int64_t n, const int32_t *rp) {
  int32_t k = 0;
  for (int64_t i = 0; i < n; ++i) {
    int32_t len = rp[i + 1] - rp[i];
    if (len > k) k = len;
  }
  return k;
}

/* ELL: entry k of row i at k*stride + i; padding col = -1, val = +0.0. */
void or_csr_to_ell(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                   int32_t K, int64_t stride, int32_t *ecol, double *eval) {
  for (int64_t s = 0; s < (int64_t)K * stride; ++s) {
    ecol[s] = -1;
    eval[s] = 0.0;
  }
  for (int64_t i = 0; i < n; ++i) {
    int32_t len = rp[i + 1] - rp[i];
    for (int32_t k = 0; k < len && k < K; ++k) {
      ecol[(int64_t)k * stride + i] = col[rp[i] + k];
      eval[(int64_t)k * stride + i] = val[rp[i] + k];
    }
  }
}

void or_spmv_ell(int64_t n, int32_t K, int64_t stride, const int32_t *ecol, const double *eval,
                 const double *x, double alpha, double beta, double *y) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int32_t k = 0; k < K; ++k) {
      int32_t c = ecol[(int64_t)k * stride + i];
      if (c >= 0) s += eval[(int64_t)k * stride + i] * x[c];
    }
    y[i] = beta == 0.0 ? alpha * s : alpha * s + beta * y[i];
  }
}

/* SELL-P (sliced ELL with padding; the Sellp format of Section 1 and the
 * SpMV of Section 4, layout as defined by Anzt, Tomov & Dongarra, "Implementing
 * a sparse matrix vector product for the SELL-C/SELL-P format on NVIDIA GPUs",
 * 2014): rows are cut into slices of C consecutive rows (no reordering); slice
 * s is as wide as its longest row, w_s, and holds its entries column-major:
 * entry k of row i (slice s = i / C) sits at (sets[s] + k) * C + i % C, with
 * sets[s] = w_0 + ... + w_{s-1}.  Padding col = -1, val = +0.0. */
int64_t or_sellp_slices(int64_t n, int32_t C) { return (n + C - 1) / C; }

/* sets[0..n_slices]: prefix sums of the slice widths; returns sets[n_slices]. */
int64_t or_sellp_sets(int64_t n, const int32_t *rp, int32_t C, int64_t *sets) {
  int64_t ns = or_sellp_slices(n, C);
  sets[0] = 0;
  for (int64_t sl = 0; sl < ns; ++sl) {
    int32_t w = 0;
    for (int64_t i = sl * C; i < n && i < (sl + 1) * C; ++i) {
      int32_t len = rp[i + 1] - rp[i];
      if (len > w) w = len;
    }
    sets[sl + 1] = sets[sl] + w;
  }
  return sets[ns];
}

void or_csr_to_sellp(int64_t n, const int32_t *rp, const int32_t *col, const double *val, int32_t C,
                     const int64_t *sets, int32_t *scol, double *sval) {
  int64_t ns = or_sellp_slices(n, C);
  for (int64_t q = 0; q < sets[ns] * C; ++q) {
    scol[q] = -1;
    sval[q] = 0.0;
  }
  for (int64_t i = 0; i < n; ++i) {
    int64_t sl = i / C;
    for (int32_t k = 0; k < rp[i + 1] - rp[i]; ++k) {
      int64_t q = (sets[sl] + k) * C + i % C;
      scol[q] = col[rp[i] + k];
      sval[q] = val[rp[i] + k];
    }
  }
}

void or_spmv_sellp(int64_t n, int32_t C, const int64_t *sets, const int32_t *scol, const double *sval,
                   const double *x, double alpha, double beta, double *y) {
  for (int64_t i = 0; i < n; ++i) {
    int64_t sl = i / C;
    double s = 0.0;
    for (int64_t k = 0; k < sets[sl + 1] - sets[sl]; ++k) {
      int64_t q = (sets[sl] + k) * C + i % C;
      if (scol[q] >= 0) s += sval[q] * x[scol[q]];
    }
    y[i] = beta == 0.0 ? alpha * s : alpha * s + beta * y[i];
  }
}

/* Subwarp butterfly reduction of the paper's Section 3.3 benchmark (the
 * reduce listing): lanes are grouped into subwarps of S consecutive lanes
 * (S divides 32); each of `loops` rounds runs log2(S) steps in which every
 * lane adds the value of the lane whose index differs in bit `bitmask`
 * (bitmask = 1, 2, ..., S/2), all lanes of a step reading the values of the
 * previous step.  n must be a multiple of S. */
void or_subwarp_reduce(int64_t n, int32_t S, int32_t loops, double *data) {
  double *tmp = (double *)malloc(sizeof(double) * (size_t)(S > 0 ? S : 1));
  for (int64_t g = 0; g + S <= n; g += S)
    for (int32_t it = 0; it < loops; ++it)
      for (int32_t bitmask = 1; bitmask < S; bitmask <<= 1) {
        for (int32_t l = 0; l < S; ++l) tmp[l] = data[g + l] + data[g + (l ^ bitmask)];
        for (int32_t l = 0; l < S; ++l) data[g + l] = tmp[l];
      }
  free(tmp);
}

/* COO: row-major expansion of CSR in storage order. */
void or_csr_to_coo(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                   int32_t *crow, int32_t *ccol, double *cval) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      crow[k] = (int32_t)i;
      ccol[k] = col[k];
      cval[k] = val[k];
    }
}

/* COO SpMV: per-row sums accumulated in entry order, then scaled.  The
 * temporary t is the plain definition's per-row accumulator. */
int or_spmv_coo(int64_t n, int64_t nnz, const int32_t *crow, const int32_t *ccol,
                const double *cval, const double *x, double alpha, double beta, double *y) {
  double *t = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  if (!t) return OR_INVALID;
  for (int64_t k = 0; k < nnz; ++k) t[crow[k]] += cval[k] * x[ccol[k]];
  for (int64_t i = 0; i < n; ++i) y[i] = beta == 0.0 ? alpha * t[i] : alpha * t[i] + beta * y[i];
  free(t);
  return OR_OK;
}

/* Hybrid width: largest k with count(len >= k) >= max(4096, n/3). */
int32_t or_hybrid_width(int64_t n, const int32_t *rp) {
  int32_t maxlen = or_ell_width(n, rp);
  int64_t *cnt = (int64_t *)calloc((size_t)maxlen + 2, sizeof(int64_t));
  if (!cnt) return -1;
  for (int64_t i = 0; i < n; ++i) cnt[rp[i + 1] - rp[i]] += 1;
  /* turn the histogram into suffix counts: cnt[k] = #{len >= k} */
  for (int64_t k = maxlen - 1; k >= 0; --k) cnt[k] += cnt[k + 1];
  int32_t K = 0;
  for (int32_t k = 0; k <= maxlen; ++k)
    if (cnt[k] >= 4096 && 3 * cnt[k] >= n) K = k;
  free(cnt);
  return K;
}

/* Number of COO entries in the hybrid tail for width K. */
int64_t or_hybrid_tail_nnz(int64_t n, const int32_t *rp, int32_t K) {
  int64_t t = 0;
  for (int64_t i = 0; i < n; ++i) {
    int32_t len = rp[i + 1] - rp[i];
    if (len > K) t += len - K;
  }
  return t;
}

/* Hybrid: the first min(len, K) entries of each row go to ELL (width K),
 * the rest to a row-major COO tail, both in storage order. */
void or_csr_to_hybrid(int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                      int32_t K, int64_t stride, int32_t *ecol, double *eval, int32_t *crow,
                      int32_t *ccol, double *cval) {
  or_csr_to_ell(n, rp, col, val, K, stride, ecol, eval);
  int64_t t = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = rp[i] + K; k < rp[i + 1]; ++k) {
      crow[t] = (int32_t)i;
      ccol[t] = col[k];
      cval[t] = val[k];
      ++t;
    }
}

/* Hybrid SpMV: each row adds its ELL entries then its COO entries, i.e. the
 * CSR storage order. */
int or_spmv_hybrid(int64_t n, int32_t K, int64_t stride, const int32_t *ecol, const double *eval,
                   int64_t tail, const int32_t *crow, const int32_t *ccol, const double *cval,
                   const double *x, double alpha, double beta, double *y) {
  double *t = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  if (!t) return OR_INVALID;
  for (int64_t i = 0; i < n; ++i)
    for (int32_t k = 0; k < K; ++k) {
      int32_t c = ecol[(int64_t)k * stride + i];
      if (c >= 0) t[i] += eval[(int64_t)k * stride + i] * x[c];
    }
  for (int64_t k = 0; k < tail; ++k) t[crow[k]] += cval[k] * x[ccol[k]];
  for (int64_t i = 0; i < n; ++i) y[i] = beta == 0.0 ? alpha * t[i] : alpha * t[i] + beta * y[i];
  free(t);
  return OR_OK;
}

/* -------------------------------------------------------------- BLAS-1 -- */

/* Sequential FP64 definitions of the vector operations inside the Krylov
 * solvers: dot = sum_i x_i y_i (left to right); axpy y_i = a x_i + y_i;
 * multi-dot h_j = V_j . w; multi-axpy + norm y -= sum_j h_j V_j (j in
 * order for each i), then ||y||_2. */
double or_dot(int64_t n, const double *x, const double *y) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
  return s;
}

void or_axpy(int64_t n, double a, const double *x, double *y) {
  for (int64_t i = 0; i < n; ++i) y[i] = a * x[i] + y[i];
}

void or_multi_dot(int64_t n, int32_t k, const double *V, int64_t ldv, const double *w, double *h) {
  for (int32_t j = 0; j < k; ++j) h[j] = or_dot(n, V + (int64_t)j * ldv, w);
}

double or_multi_axpy_norm(int64_t n, int32_t k, const double *h, const double *V, int64_t ldv, double *y) {
  for (int64_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < k; ++j) y[i] = y[i] - h[j] * V[(int64_t)j * ldv + i];
  return sqrt(or_dot(n, y, y));
}

/* ------------------------------------------------------------- solvers -- */

/* A CSR operator: FP64 values, or FP32 values with FP32 accumulation (the
 * inner operator of mixed-precision refinement). */
typedef struct {
  int64_t n;
  const int32_t *rp, *col;
  const double *val;
  const float *val32;
} or_op;

/* y = A x.  With FP32 values: the FP32 SpMV above on fl32(x), widened. */
static void op_apply(const or_op *A, const double *x, double *y) {
  if (A->val32) {
    float *xs = (float *)malloc(sizeof(float) * (size_t)(A->n + 1));
    float *ys = (float *)malloc(sizeof(float) * (size_t)(A->n + 1));
    for (int64_t i = 0; i < A->n; ++i) xs[i] = (float)x[i];
    or_spmv_csr_f32(A->n, A->rp, A->col, A->val32, xs, 1.0f, 0.0f, ys);
    for (int64_t i = 0; i < A->n; ++i) y[i] = (double)ys[i];
    free(xs);
    free(ys);
  } else {
    /* the plain CSR SpMV above (rows over the OpenMP threads, each row summed
     * in storage order; alpha = 1 gives y = s exactly) */
    or_spmv_csr(A->n, A->rp, A->col, A->val, x, 1.0, 0.0, y);
  }
}

/* Storage rounding of a vector element: FP32 for the inner solve of the
 * mixed-precision refinement, identity otherwise. */
static inline double st(int f32, double v) { return f32 ? (double)(float)v : v; }

static double dot(int64_t n, const double *a, const double *b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static double nrm2(int64_t n, const double *a) { return sqrt(dot(n, a, a)); }

/* r = b - A x (FP64 storage) */
static void residual(const or_op *A, const double *b, const double *x, double *r, double *tmp) {
  op_apply(A, x, tmp);
  for (int64_t i = 0; i < A->n; ++i) r[i] = b[i] - tmp[i];
}

typedef struct {
  int32_t status;
  int32_t iterations;
  int32_t outer_iterations;
  int32_t pad;
  double rel_residual;
} or_result;

/* Common solver context: A, the storage rounding flag, whether to verify a
 * converged recurrence residual against the true residual, and an optional
 * per-iteration history of ||r||/||b|| (recurrence or Givens estimate). */
typedef struct {
  const or_op *A;
  int f32;
  int true_check;
  double *hist;
  int32_t hist_len;
  const double *minv; /* Jacobi preconditioner: inverse diagonal, or NULL */
  const double *bj;   /* block-Jacobi: inverse diagonal blocks (or_block_jacobi_inv), or NULL */
  int32_t bs;         /* block-Jacobi block size */
} or_ctx;

/* z = M^-1 r for the Jacobi preconditioner M = diag(A) (Saad, Sec. 10.2),
 * or for block-Jacobi M = the block diagonal of A (Saad, Sec. 12.2): row i
 * of block k (rows k*bs .. k*bs + nb - 1) takes z_i = sum_j B[i*bs + j] *
 * r[k*bs + j], j = 0 .. nb - 1 in order; the identity without either. */
static void precond(const or_ctx *c, const double *r, double *z) {
  const int64_t n = c->A->n;
  if (c->bj) {
    for (int64_t i = 0; i < n; ++i) {
      const int64_t base = i / c->bs * c->bs;
      const int64_t nb = n - base < c->bs ? n - base : c->bs;
      double s = 0.0;
      for (int64_t j = 0; j < nb; ++j) s += c->bj[i * c->bs + j] * r[base + j];
      z[i] = st(c->f32, s);
    }
    return;
  }
  for (int64_t i = 0; i < n; ++i) z[i] = c->minv ? st(c->f32, c->minv[i] * r[i]) : r[i];
}

/* Inverse diagonal of a CSR matrix: diagonal entries of a row summed in
 * storage order (duplicates add up as in the SpMV); a zero or missing
 * diagonal gives 1 (that row is left unscaled). */
void or_jacobi_inv(int64_t n, const int32_t *rp, const int32_t *col, const double *val, double *minv) {
  for (int64_t i = 0; i < n; ++i) {
    double d = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
      if (col[k] == i) d += val[k];
    minv[i] = d != 0.0 ? 1.0 / d : 1.0;
  }
}

/* Block-Jacobi setup (Saad, Sec. 12.2): the diagonal blocks of A are rows
 * and columns k*bs .. k*bs + nb - 1 with nb = min(bs, n - k*bs) (the last
 * block may be smaller).  Each block is gathered densely (entries of a row
 * summed in storage order, so duplicates add up as in the SpMV) and inverted
 * by Gauss-Jordan elimination on [D | I] with partial pivoting (pivot: the
 * first row of largest magnitude in the column; the pivot row multiplied
 * by the reciprocal of the pivot, one division per step, as Golub & Van
 * Loan scale it; then every other row r takes row_r - m_r * row_k with m_r
 * its entry in the pivot column).  A block whose pivot column is all zero at
 * some step is singular and is replaced by the identity (its rows are left
 * unscaled, as a zero diagonal is for Jacobi).  Output: row i of the inverse
 * at B[i*bs .. i*bs + nb - 1], zeros in B[i*bs + nb .. i*bs + bs - 1].
 * Returns the number of singular blocks; bs must lie in 1..64. */
int64_t or_block_jacobi_inv(int64_t n, const int32_t *rp, const int32_t *col, const double *val, int32_t bs,
                            double *B) {
  if (bs < 1 || bs > 64) return -1;
  double *M = malloc(sizeof(double) * (size_t)bs * 2 * (size_t)bs);
  int64_t singular = 0;
  for (int64_t base = 0; base < n; base += bs) {
    const int64_t nb = n - base < bs ? n - base : bs;
    const int64_t w = 2 * nb;
    for (int64_t r = 0; r < nb; ++r) {
      for (int64_t c = 0; c < w; ++c) M[r * w + c] = 0.0;
      M[r * w + nb + r] = 1.0;
      for (int64_t k = rp[base + r]; k < rp[base + r + 1]; ++k) {
        const int64_t c = (int64_t)col[k] - base;
        if (c >= 0 && c < nb) M[r * w + c] += val[k];
      }
    }
    int ok = 1;
    for (int64_t k = 0; k < nb && ok; ++k) {
      int64_t piv = k;
      for (int64_t r = k + 1; r < nb; ++r)
        if (fabs(M[r * w + k]) > fabs(M[piv * w + k])) piv = r;
      if (M[piv * w + k] == 0.0) {
        ok = 0;
        break;
      }
      if (piv != k)
        for (int64_t c = 0; c < w; ++c) {
          const double t = M[k * w + c];
          M[k * w + c] = M[piv * w + c];
          M[piv * w + c] = t;
        }
      const double inv = 1.0 / M[k * w + k];
      for (int64_t c = 0; c < w; ++c) M[k * w + c] = M[k * w + c] * inv;
      for (int64_t r = 0; r < nb; ++r) {
        if (r == k) continue;
        const double m = M[r * w + k];
        for (int64_t c = 0; c < w; ++c) M[r * w + c] = M[r * w + c] - m * M[k * w + c];
      }
    }
    for (int64_t r = 0; r < nb; ++r)
      for (int64_t j = 0; j < bs; ++j)
        B[(base + r) * bs + j] = j < nb ? (ok ? M[r * w + nb + j] : (r == j ? 1.0 : 0.0)) : 0.0;
    if (!ok) ++singular;
  }
  free(M);
  return singular;
}

static void hist_put(const or_ctx *c, int32_t it, double v) {
  if (c->hist && it >= 1 && it <= c->hist_len) c->hist[it - 1] = v;
}

/* CG (Saad Alg. 6.18), or preconditioned CG with z = M^-1 r (Saad Alg.
 * 9.1) when c->minv is set; convergence is always judged on ||r||.  x holds
 * x0 on entry and the iterate on exit. */
static or_result cg_core(const or_ctx *c, const double *b, double *x, double tol, int32_t maxit) {
  const or_op *A = c->A;
  int64_t n = A->n;
  or_result res = {OR_OK, 0, 0, 0, 0.0};
  double *r = calloc((size_t)n + 1, sizeof(double)), *p = calloc((size_t)n + 1, sizeof(double));
  double *q = calloc((size_t)n + 1, sizeof(double)), *t = calloc((size_t)n + 1, sizeof(double));
  double *z = calloc((size_t)n + 1, sizeof(double));
  double nb = nrm2(n, b);
  if (nb == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    goto done;
  }
  residual(A, b, x, r, t);
  for (int64_t i = 0; i < n; ++i) r[i] = st(c->f32, r[i]);
  precond(c, r, z);
  for (int64_t i = 0; i < n; ++i) p[i] = z[i];
  double rho = dot(n, r, z);
  int converged = nrm2(n, r) <= tol * nb;
  int32_t it = 0;
  while (!converged && it < maxit) {
    op_apply(A, p, q);
    for (int64_t i = 0; i < n; ++i) q[i] = st(c->f32, q[i]);
    double pq = dot(n, p, q);
    if (!(pq > 0.0)) {
      res.status = OR_BREAKDOWN;
      break;
    }
    double alpha = rho / pq;
    for (int64_t i = 0; i < n; ++i) {
      x[i] = st(c->f32, x[i] + alpha * p[i]);
      r[i] = st(c->f32, r[i] - alpha * q[i]);
    }
    double nr = nrm2(n, r);
    ++it;
    hist_put(c, it, nr / nb);
    if (nr <= tol * nb) {
      if (!c->true_check) {
        converged = 1;
        break;
      }
      residual(A, b, x, t, q);
      if (nrm2(n, t) <= tol * nb) {
        converged = 1;
        break;
      }
      for (int64_t i = 0; i < n; ++i) r[i] = t[i]; /* residual replacement */
    }
    precond(c, r, z);
    double rho_new = dot(n, r, z);
    double beta = rho_new / rho;
    for (int64_t i = 0; i < n; ++i) p[i] = st(c->f32, z[i] + beta * p[i]);
    rho = rho_new;
  }
  res.iterations = it;
  if (res.status == OR_OK && !converged) res.status = OR_NOT_CONVERGED;
done:
  if (nb == 0.0) {
    res.rel_residual = 0.0;
  } else {
    residual(A, b, x, r, t);
    res.rel_residual = nrm2(n, r) / nb;
  }
  free(r);
  free(p);
  free(q);
  free(t);
  free(z);
  return res;
}

/* BiCGSTAB (van der Vorst 1992; Saad Alg. 7.7); with c->minv the right
 * preconditioned form: the products are A (M^-1 p) and A (M^-1 s), and x
 * moves along M^-1 p and M^-1 s. */
static or_result bicgstab_core(const or_ctx *c, const double *b, double *x, double tol,
                               int32_t maxit) {
  const or_op *A = c->A;
  int64_t n = A->n;
  or_result res = {OR_OK, 0, 0, 0, 0.0};
  size_t sz = (size_t)n + 1;
  double *r = calloc(sz, 8), *rh = calloc(sz, 8), *p = calloc(sz, 8), *v = calloc(sz, 8);
  double *s = calloc(sz, 8), *t = calloc(sz, 8), *w = calloc(sz, 8);
  double *ph = calloc(sz, 8), *sh = calloc(sz, 8);
  double nb = nrm2(n, b);
  int converged = 0;
  int32_t it = 0;
  if (nb == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    goto done;
  }
  residual(A, b, x, r, w);
  for (int64_t i = 0; i < n; ++i) r[i] = rh[i] = st(c->f32, r[i]);
  double rho = 1.0, alpha = 1.0, omega = 1.0;
  converged = nrm2(n, r) <= tol * nb;
  while (!converged && it < maxit) {
    double rho_new = dot(n, rh, r);
    if (rho_new == 0.0) {
      res.status = OR_BREAKDOWN;
      break;
    }
    double beta = (rho_new / rho) * (alpha / omega);
    for (int64_t i = 0; i < n; ++i) p[i] = st(c->f32, r[i] + beta * (p[i] - omega * v[i]));
    precond(c, p, ph);
    op_apply(A, ph, v);
    for (int64_t i = 0; i < n; ++i) v[i] = st(c->f32, v[i]);
    double rv = dot(n, rh, v);
    if (rv == 0.0) {
      res.status = OR_BREAKDOWN;
      break;
    }
    alpha = rho_new / rv;
    for (int64_t i = 0; i < n; ++i) s[i] = st(c->f32, r[i] - alpha * v[i]);
    ++it;
    int restart = 0;
    if (nrm2(n, s) <= tol * nb) {
      for (int64_t i = 0; i < n; ++i) x[i] = st(c->f32, x[i] + alpha * ph[i]);
      hist_put(c, it, nrm2(n, s) / nb);
      if (!c->true_check) {
        converged = 1;
        break;
      }
      residual(A, b, x, w, t);
      if (nrm2(n, w) <= tol * nb) {
        converged = 1;
        break;
      }
      restart = 1;
    } else {
      precond(c, s, sh);
      op_apply(A, sh, t);
      for (int64_t i = 0; i < n; ++i) t[i] = st(c->f32, t[i]);
      double tt = dot(n, t, t);
      if (tt == 0.0) {
        res.status = OR_BREAKDOWN;
        break;
      }
      omega = dot(n, t, s) / tt;
      for (int64_t i = 0; i < n; ++i) {
        x[i] = st(c->f32, x[i] + alpha * ph[i] + omega * sh[i]);
        r[i] = st(c->f32, s[i] - omega * t[i]);
      }
      rho = rho_new;
      double nr = nrm2(n, r);
      hist_put(c, it, nr / nb);
      if (nr <= tol * nb) {
        if (!c->true_check) {
          converged = 1;
          break;
        }
        residual(A, b, x, w, t);
        if (nrm2(n, w) <= tol * nb) {
          converged = 1;
          break;
        }
        restart = 1;
      } else if (omega == 0.0) {
        res.status = OR_BREAKDOWN;
        break;
      }
    }
    if (restart) { /* residual replacement restarts the recurrences */
      for (int64_t i = 0; i < n; ++i) {
        r[i] = w[i];
        p[i] = v[i] = 0.0;
      }
      rho = alpha = omega = 1.0;
    }
  }
  res.iterations = it;
  if (res.status == OR_OK && !converged) res.status = OR_NOT_CONVERGED;
done:
  if (nb == 0.0) {
    res.rel_residual = 0.0;
  } else {
    residual(A, b, x, r, w);
    res.rel_residual = nrm2(n, r) / nb;
  }
  free(r);
  free(rh);
  free(p);
  free(v);
  free(s);
  free(t);
  free(w);
  free(ph);
  free(sh);
  return res;
}

/* Restarted GMRES(m) with modified Gram-Schmidt and Givens rotations
 * (Saad & Schultz 1986; Saad Alg. 6.9 and 6.11).  Iterations count Arnoldi
 * steps; each cycle starts from the true residual. */
static or_result gmres_core(const or_ctx *c, const double *b, double *x, double tol,
                            int32_t maxit, int32_t m) {
  const or_op *A = c->A;
  int64_t n = A->n;
  or_result res = {OR_OK, 0, 0, 0, 0.0};
  if (m < 1) m = 1;
  size_t sz = (size_t)n + 1;
  double *V = calloc(sz * (size_t)(m + 1), 8);
  double *H = calloc((size_t)(m + 1) * (size_t)m, 8); /* H[i*m + j] = h_{i,j} */
  double *cs = calloc((size_t)m, 8), *sn = calloc((size_t)m, 8);
  double *g = calloc((size_t)m + 1, 8), *yv = calloc((size_t)m, 8);
  double *r = calloc(sz, 8), *w = calloc(sz, 8), *tmp = calloc(sz, 8);
  double nb = nrm2(n, b);
  int converged = 0;
  int32_t it = 0;
  if (nb == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    goto done;
  }
  for (;;) {
    residual(A, b, x, r, tmp);
    for (int64_t i = 0; i < n; ++i) r[i] = st(c->f32, r[i]);
    double beta = nrm2(n, r);
    if (beta <= tol * nb) {
      converged = 1;
      break;
    }
    if (it >= maxit) break;
    for (int64_t i = 0; i < n; ++i) V[i] = st(c->f32, r[i] / beta);
    memset(g, 0, sizeof(double) * (size_t)(m + 1));
    g[0] = beta;
    int32_t k = 0;
    int stop = 0;
    for (int32_t j = 0; j < m && it < maxit; ++j) {
      double *vj = V + (size_t)j * sz;
      op_apply(A, vj, w);
      for (int64_t i = 0; i < n; ++i) w[i] = st(c->f32, w[i]);
      for (int32_t i = 0; i <= j; ++i) {
        double *vi = V + (size_t)i * sz;
        double h = dot(n, w, vi);
        H[(size_t)i * m + j] = h;
        for (int64_t e = 0; e < n; ++e) w[e] = st(c->f32, w[e] - h * vi[e]);
      }
      double hn = nrm2(n, w);
      H[(size_t)(j + 1) * m + j] = hn;
      for (int32_t i = 0; i < j; ++i) {
        double a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      double a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
      double den = sqrt(a * a + bb * bb);
      ++it;
      k = j + 1;
      if (den == 0.0) {
        res.status = OR_BREAKDOWN;
        k = j;
        stop = 2;
        break;
      }
      cs[j] = a / den;
      sn[j] = bb / den;
      H[(size_t)j * m + j] = den;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      hist_put(c, it, fabs(g[j + 1]) / nb);
      if (hn == 0.0 || fabs(g[j + 1]) <= tol * nb) {
        stop = 1;
        break;
      }
      double *vn = V + (size_t)(j + 1) * sz;
      for (int64_t i = 0; i < n; ++i) vn[i] = st(c->f32, w[i] / hn);
    }
    /* back substitution H[0:k,0:k] y = g[0:k], then x += V y */
    for (int32_t i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int32_t l = i + 1; l < k; ++l) s -= H[(size_t)i * m + l] * yv[l];
      yv[i] = s / H[(size_t)i * m + i];
    }
    for (int64_t e = 0; e < n; ++e) {
      double s = 0.0;
      for (int32_t i = 0; i < k; ++i) s += V[(size_t)i * sz + e] * yv[i];
      x[e] = st(c->f32, x[e] + s);
    }
    res.outer_iterations += 1;
    if (stop == 2) break;
    if (stop == 1 && !c->true_check) {
      converged = 1;
      break;
    }
  }
  res.iterations = it;
  if (res.status == OR_OK && !converged) res.status = OR_NOT_CONVERGED;
done:
  if (nb == 0.0) {
    res.rel_residual = 0.0;
  } else {
    residual(A, b, x, r, tmp);
    res.rel_residual = nrm2(n, r) / nb;
  }
  free(V);
  free(H);
  free(cs);
  free(sn);
  free(g);
  free(yv);
  free(r);
  free(w);
  free(tmp);
  return res;
}

enum { OR_SOLVER_CG = 0, OR_SOLVER_BICGSTAB = 1, OR_SOLVER_GMRES = 2 };

static or_result run_solver(const or_ctx *c, int solver, const double *b, double *x, double tol,
                            int32_t maxit, int32_t restart) {
  if (solver == OR_SOLVER_CG) return cg_core(c, b, x, tol, maxit);
  if (solver == OR_SOLVER_BICGSTAB) return bicgstab_core(c, b, x, tol, maxit);
  return gmres_core(c, b, x, tol, maxit, restart);
}

/* FP64 Krylov solve.  x: x0 on entry, the solution on exit.  hist (optional,
 * hist_len entries) receives ||r_k||/||b|| per iteration. */
int or_solve(int solver, int64_t n, const int32_t *rp, const int32_t *col, const double *val,
             const double *b, double *x, double tol, int32_t maxit, int32_t restart,
             double *hist, int32_t hist_len, or_result *out) {
  or_op A = {n, rp, col, val, NULL};
  or_ctx c = {&A, 0, 1, hist, hist_len, NULL};
  *out = run_solver(&c, solver, b, x, tol, maxit, restart);
  return out->status;
}

/* Jacobi-preconditioned FP64 CG / BiCGSTAB (minv: the inverse diagonal from
 * or_jacobi_inv).  GMRES is not offered with a preconditioner (OR_INVALID). */
int or_solve_pc(int solver, int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                const double *minv, const double *b, double *x, double tol, int32_t maxit, or_result *out) {
  or_result bad = {OR_INVALID, 0, 0, 0, 0.0};
  if (solver != OR_SOLVER_CG && solver != OR_SOLVER_BICGSTAB) {
    *out = bad;
    return OR_INVALID;
  }
  or_op A = {n, rp, col, val, NULL};
  or_ctx c = {&A, 0, 1, NULL, 0, minv};
  *out = run_solver(&c, solver, b, x, tol, maxit, 0);
  return out->status;
}

/* Block-Jacobi-preconditioned FP64 CG / BiCGSTAB (B, bs: the inverse
 * diagonal blocks from or_block_jacobi_inv).  GMRES: OR_INVALID. */
int or_solve_bj(int solver, int64_t n, const int32_t *rp, const int32_t *col, const double *val, int32_t bs,
                const double *B, const double *b, double *x, double tol, int32_t maxit, or_result *out) {
  or_result bad = {OR_INVALID, 0, 0, 0, 0.0};
  if ((solver != OR_SOLVER_CG && solver != OR_SOLVER_BICGSTAB) || bs < 1) {
    *out = bad;
    return OR_INVALID;
  }
  or_op A = {n, rp, col, val, NULL};
  or_ctx c = {&A, 0, 1, NULL, 0, NULL, B, bs};
  *out = run_solver(&c, solver, b, x, tol, maxit, 0);
  return out->status;
}

/* Batched CG (the single-system CG above applied to each system on its own):
 * system i has rows [row_off[i], row_off[i+1]) of b and x, local row
 * pointers starting at rp[row_off[i] + i] and entries [nnz_off[i],
 * nnz_off[i+1]) of col/val.  Systems are spread over the OpenMP threads;
 * each system's solve is sequential, so results do not depend on the
 * thread count.  iters, relres, status: per system. */
void or_batch_cg(int32_t count, const int64_t *row_off, const int64_t *nnz_off, const int32_t *rp,
                 const int32_t *col, const double *val, const double *b, double *x, double tol, int32_t maxit,
                 int32_t *iters, double *relres, int32_t *status) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
#endif
  for (int32_t i = 0; i < count; ++i) {
    const int64_t r0 = row_off[i], k0 = nnz_off[i];
    or_op A = {row_off[i + 1] - r0, rp + r0 + i, col + k0, val + k0, NULL};
    or_ctx c = {&A, 0, 1, NULL, 0, NULL};
    const or_result res = cg_core(&c, b + r0, x + r0, tol, maxit);
    iters[i] = res.iterations;
    relres[i] = res.rel_residual;
    status[i] = res.status;
  }
}

/* Mixed-precision iterative refinement: x = x0; repeat { r = b - A64 x in
 * FP64; stop if ||r|| <= tol ||b||; solve A32 d = r with FP32-stored values
 * and vectors (FP32 SpMV accumulation, FP64 dots and scalars) to
 * ||r_inner|| <= inner_tol ||r|| (adaptive != 0: to max(inner_tol, min(0.5,
 * 0.5 tol ||b|| / ||r||)) ||r||, the library's adaptive tunable); x += d in
 * FP64 }. */
static int solve_ir(int solver, int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                    const float *val32, const double *minv, const double *bj, int32_t bs, const double *b,
                    double *x, double tol, int32_t max_outer, double inner_tol, int32_t inner_maxit,
                    int32_t restart, int adaptive, or_result *out);

int or_solve_ir(int solver, int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                const float *val32, const double *b, double *x, double tol, int32_t max_outer,
                double inner_tol, int32_t inner_maxit, int32_t restart, int32_t adaptive, or_result *out) {
  return solve_ir(solver, n, rp, col, val, val32, NULL, NULL, 0, b, x, tol, max_outer, inner_tol, inner_maxit,
                  restart, adaptive, out);
}

/* Mixed-precision refinement whose inner CG / BiCGSTAB is Jacobi
 * preconditioned with the FP64 inverse diagonal rounded to FP32 (the inner
 * solve stores everything in FP32). */
int or_solve_ir_pc(int solver, int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                   const float *val32, const double *minv, const double *b, double *x, double tol,
                   int32_t max_outer, double inner_tol, int32_t inner_maxit, int32_t adaptive, or_result *out) {
  if (solver != OR_SOLVER_CG && solver != OR_SOLVER_BICGSTAB) {
    or_result bad = {OR_INVALID, 0, 0, 0, 0.0};
    *out = bad;
    return OR_INVALID;
  }
  return solve_ir(solver, n, rp, col, val, val32, minv, NULL, 0, b, x, tol, max_outer, inner_tol, inner_maxit, 0,
                  adaptive, out);
}

/* Mixed-precision refinement whose inner CG / BiCGSTAB is block-Jacobi
 * preconditioned with the FP64 inverse blocks (or_block_jacobi_inv) rounded
 * to FP32. */
int or_solve_ir_bj(int solver, int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                   const float *val32, int32_t bs, const double *B, const double *b, double *x, double tol,
                   int32_t max_outer, double inner_tol, int32_t inner_maxit, int32_t adaptive, or_result *out) {
  if ((solver != OR_SOLVER_CG && solver != OR_SOLVER_BICGSTAB) || bs < 1) {
    or_result bad = {OR_INVALID, 0, 0, 0, 0.0};
    *out = bad;
    return OR_INVALID;
  }
  return solve_ir(solver, n, rp, col, val, val32, NULL, B, bs, b, x, tol, max_outer, inner_tol, inner_maxit, 0,
                  adaptive, out);
}

/* fl32 copy of a preconditioner array (as doubles), or NULL */
static double *round32_copy(const double *a, int64_t count) {
  if (!a) return NULL;
  double *m = calloc((size_t)count + 1, 8);
  for (int64_t i = 0; i < count; ++i) m[i] = (double)(float)a[i];
  return m;
}

static int solve_ir(int solver, int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                    const float *val32, const double *minv, const double *bj, int32_t bs, const double *b,
                    double *x, double tol, int32_t max_outer, double inner_tol, int32_t inner_maxit,
                    int32_t restart, int adaptive, or_result *out) {
  or_op A64 = {n, rp, col, val, NULL};
  or_op A32 = {n, rp, col, NULL, val32};
  size_t sz = (size_t)n + 1;
  double *minv32 = round32_copy(minv, n);
  double *bj32 = round32_copy(bj, n * (int64_t)bs);
  or_ctx inner = {&A32, 1, 0, NULL, 0, minv32, bj32, bs};
  or_result res = {OR_OK, 0, 0, 0, 0.0};
  double *r = calloc(sz, 8), *d = calloc(sz, 8), *tmp = calloc(sz, 8);
  double nb = nrm2(n, b);
  int converged = 0;
  if (nb == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    converged = 1;
  }
  while (!converged) {
    residual(&A64, b, x, r, tmp);
    double nr = nrm2(n, r);
    if (nr <= tol * nb) {
      converged = 1;
      break;
    }
    if (res.outer_iterations >= max_outer) break;
    for (int64_t i = 0; i < n; ++i) d[i] = 0.0;
    /* the inner solve reduces the residual by the fixed factor inner_tol
     * (refinement with an inner solver of fixed relative accuracy, as in
     * Carson & Higham 2018).  adaptive: the library's tunable instead, which
     * asks only for the reduction still needed, with a factor-2 margin:
     * max(inner_tol, min(0.5, 0.5 * tol * ||b|| / ||r||)). */
    double itol = inner_tol;
    if (adaptive) {
      double need = 0.5 * tol * nb / nr;
      if (need > 0.5) need = 0.5;
      itol = need > inner_tol ? need : inner_tol;
    }
    or_result in = run_solver(&inner, solver, r, d, itol, inner_maxit, restart);
    res.iterations += in.iterations;
    res.outer_iterations += 1;
    for (int64_t i = 0; i < n; ++i) x[i] += d[i];
  }
  if (!converged) res.status = OR_NOT_CONVERGED;
  if (nb == 0.0) {
    res.rel_residual = 0.0;
  } else {
    residual(&A64, b, x, r, tmp);
    res.rel_residual = nrm2(n, r) / nb;
  }
  free(r);
  free(d);
  free(tmp);
  free(minv32);
  free(bj32);
  *out = res;
  return res.status;
}

/* ------------------------------------------- reliable-update refinement -- */

/* Mixed precision with reliable updates: the Krylov recurrences of CG or
 * BiCGSTAB run on the inner operator (FP32 values with FP32 accumulation
 * when val32 is given, else the FP64 matrix) with every vector stored in the
 * inner precision (f32 != 0: rounded to FP32), FP64 dots and FP64 scalars;
 * the iterate's change since the last update is kept in y.  When the
 * recurrence residual drops to tol ||b||, or below delta times its largest
 * value since the last update, an update folds y into the FP64 solution x
 * (x += y, y = 0), forms the FP64 residual b - A x with the FP64 matrix and
 * replaces the recurrence residual by it (rounded to the inner precision);
 * the solve has converged when that FP64 residual meets tol ||b||, and
 * otherwise the recurrences go on with their directions and scalars kept.
 * Sources: Sleijpen & van der Vorst, "Reliable updated residuals in hybrid
 * Bi-CG methods", Computing 56 (1996) (the delta criterion and the folding of
 * the partial solution); van der Vorst & Ye, SIAM J. Sci. Comput. 22 (2000)
 * (replacing the recurrence residual by the true one without restarting);
 * Clark et al., Comput. Phys. Commun. 181 (2010) (the low precision for the
 * recurrences, the high precision for x and the replaced residual).
 * Readings: BiCGSTAB's half step (||s|| <= tol ||b||: y += alpha p, update)
 * has no continuation for its s, so an unconverged half-step update restarts
 * the recurrences (p = v = 0, rho = alpha = omega = 1) as the plain solver
 * does; after an update BiCGSTAB takes rho from rhat and the replaced r (its
 * next step's beta uses it), CG takes rho = r.z of the replaced r; omega == 0
 * is a breakdown once the step's update test has passed.  outer_iterations
 * counts the updates. */
static void fold_and_replace(const or_op *A64, int f32, const double *b, double *x, double *y, double *w,
                             double *tmp, double *rn) {
  int64_t n = A64->n;
  for (int64_t i = 0; i < n; ++i) {
    x[i] += y[i];
    y[i] = 0.0;
  }
  residual(A64, b, x, w, tmp);
  *rn = nrm2(n, w);
  for (int64_t i = 0; i < n; ++i) w[i] = st(f32, w[i]);
}

static or_result reliable_core(const or_ctx *c, const or_op *A64, int solver, const double *b, double *x,
                               double tol, int32_t maxit, double delta) {
  const or_op *A = c->A;
  int64_t n = A->n;
  size_t sz = (size_t)n + 1;
  or_result res = {OR_OK, 0, 0, 0, 0.0};
  double *y = calloc(sz, 8), *r = calloc(sz, 8), *w = calloc(sz, 8), *tmp = calloc(sz, 8);
  double *p = calloc(sz, 8), *q = calloc(sz, 8), *z = calloc(sz, 8);
  double *rh = calloc(sz, 8), *s = calloc(sz, 8), *t = calloc(sz, 8), *ph = calloc(sz, 8), *sh = calloc(sz, 8);
  double nb = nrm2(n, b), rn = 0.0;
  int converged = 0, updates = 0;
  int32_t it = 0;
  if (nb == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    converged = 1;
    goto done;
  }
  fold_and_replace(A64, c->f32, b, x, y, w, tmp, &rn);
  converged = rn <= tol * nb;
  for (int64_t i = 0; i < n; ++i) r[i] = w[i];
  double maxrr = rn;
  if (solver == OR_SOLVER_CG) {
    precond(c, r, z);
    for (int64_t i = 0; i < n; ++i) p[i] = z[i];
    double rho = dot(n, r, z);
    while (!converged && it < maxit) {
      op_apply(A, p, q);
      for (int64_t i = 0; i < n; ++i) q[i] = st(c->f32, q[i]);
      double pq = dot(n, p, q);
      if (!(pq > 0.0)) {
        res.status = OR_BREAKDOWN;
        break;
      }
      double alpha = rho / pq;
      for (int64_t i = 0; i < n; ++i) {
        y[i] = st(c->f32, y[i] + alpha * p[i]);
        r[i] = st(c->f32, r[i] - alpha * q[i]);
      }
      ++it;
      double nr = nrm2(n, r);
      hist_put(c, it, nr / nb);
      if (nr > maxrr) maxrr = nr;
      if (nr <= tol * nb || nr < delta * maxrr) {
        fold_and_replace(A64, c->f32, b, x, y, w, tmp, &rn);
        ++updates;
        if (rn <= tol * nb) {
          converged = 1;
          break;
        }
        for (int64_t i = 0; i < n; ++i) r[i] = w[i];
        maxrr = rn;
      }
      precond(c, r, z);
      double rho_new = dot(n, r, z);
      double beta = rho_new / rho;
      for (int64_t i = 0; i < n; ++i) p[i] = st(c->f32, z[i] + beta * p[i]);
      rho = rho_new;
    }
  } else {
    for (int64_t i = 0; i < n; ++i) rh[i] = r[i];
    double rho = 1.0, alpha = 1.0, omega = 1.0;
    while (!converged && it < maxit) {
      double rho_new = dot(n, rh, r);
      if (rho_new == 0.0) {
        res.status = OR_BREAKDOWN;
        break;
      }
      double beta = (rho_new / rho) * (alpha / omega);
      for (int64_t i = 0; i < n; ++i) p[i] = st(c->f32, r[i] + beta * (p[i] - omega * q[i]));
      precond(c, p, ph);
      op_apply(A, ph, q); /* q holds v = A M^-1 p */
      for (int64_t i = 0; i < n; ++i) q[i] = st(c->f32, q[i]);
      double rv = dot(n, rh, q);
      if (rv == 0.0) {
        res.status = OR_BREAKDOWN;
        break;
      }
      alpha = rho_new / rv;
      for (int64_t i = 0; i < n; ++i) s[i] = st(c->f32, r[i] - alpha * q[i]);
      ++it;
      double ns = nrm2(n, s);
      if (ns <= tol * nb) { /* half step */
        for (int64_t i = 0; i < n; ++i) y[i] = st(c->f32, y[i] + alpha * ph[i]);
        hist_put(c, it, ns / nb);
        fold_and_replace(A64, c->f32, b, x, y, w, tmp, &rn);
        ++updates;
        if (rn <= tol * nb) {
          converged = 1;
          break;
        }
        for (int64_t i = 0; i < n; ++i) {
          r[i] = w[i];
          p[i] = q[i] = 0.0;
        }
        rho = alpha = omega = 1.0;
        maxrr = rn;
        continue;
      }
      precond(c, s, sh);
      op_apply(A, sh, t);
      for (int64_t i = 0; i < n; ++i) t[i] = st(c->f32, t[i]);
      double tt = dot(n, t, t);
      if (tt == 0.0) {
        res.status = OR_BREAKDOWN;
        break;
      }
      omega = dot(n, t, s) / tt;
      for (int64_t i = 0; i < n; ++i) {
        y[i] = st(c->f32, y[i] + alpha * ph[i] + omega * sh[i]);
        r[i] = st(c->f32, s[i] - omega * t[i]);
      }
      rho = rho_new;
      double nr = nrm2(n, r);
      hist_put(c, it, nr / nb);
      if (nr > maxrr) maxrr = nr;
      if (nr <= tol * nb || nr < delta * maxrr) {
        fold_and_replace(A64, c->f32, b, x, y, w, tmp, &rn);
        ++updates;
        if (rn <= tol * nb) {
          converged = 1;
          break;
        }
        for (int64_t i = 0; i < n; ++i) r[i] = w[i];
        maxrr = rn;
      }
      if (omega == 0.0) {
        res.status = OR_BREAKDOWN;
        break;
      }
    }
  }
  for (int64_t i = 0; i < n; ++i) x[i] += y[i];
  res.iterations = it;
  res.outer_iterations = updates;
  if (res.status == OR_OK && !converged) res.status = OR_NOT_CONVERGED;
done:
  if (nb == 0.0) {
    res.rel_residual = 0.0;
  } else {
    residual(A64, b, x, w, tmp);
    res.rel_residual = nrm2(n, w) / nb;
  }
  free(y);
  free(r);
  free(w);
  free(tmp);
  free(p);
  free(q);
  free(z);
  free(rh);
  free(s);
  free(t);
  free(ph);
  free(sh);
  return res;
}

/* CG or BiCGSTAB with reliable updates (above).  val32: FP32 values for the
 * recurrences' operator (NULL: the FP64 matrix); f32: inner vectors stored
 * in FP32; minv: Jacobi inverse diagonal (NULL: none), rounded to FP32 for
 * the recurrences when f32 is set; x: x0 on entry, the solution on exit. */
int or_solve_reliable(int solver, int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                      const float *val32, const double *minv, int32_t f32, const double *b, double *x,
                      double tol, int32_t maxit, double delta, or_result *out) {
  if (solver != OR_SOLVER_CG && solver != OR_SOLVER_BICGSTAB) {
    or_result bad = {OR_INVALID, 0, 0, 0, 0.0};
    *out = bad;
    return OR_INVALID;
  }
  or_op A64 = {n, rp, col, val, NULL};
  or_op Ain = {n, rp, col, val32 ? NULL : val, val32};
  double *m = NULL;
  if (minv) {
    m = calloc((size_t)n + 1, 8);
    for (int64_t i = 0; i < n; ++i) m[i] = st(f32, minv[i]);
  }
  or_ctx c = {&Ain, f32 != 0, 0, NULL, 0, m};
  *out = reliable_core(&c, &A64, solver, b, x, tol, maxit, delta);
  free(m);
  return out->status;
}

/* The same with block-Jacobi: B, bs from or_block_jacobi_inv, rounded to
 * FP32 for the recurrences when f32 is set. */
int or_solve_reliable_bj(int solver, int64_t n, const int32_t *rp, const int32_t *col, const double *val,
                         const float *val32, int32_t bs, const double *B, int32_t f32, const double *b, double *x,
                         double tol, int32_t maxit, double delta, or_result *out) {
  if ((solver != OR_SOLVER_CG && solver != OR_SOLVER_BICGSTAB) || bs < 1) {
    or_result bad = {OR_INVALID, 0, 0, 0, 0.0};
    *out = bad;
    return OR_INVALID;
  }
  or_op A64 = {n, rp, col, val, NULL};
  or_op Ain = {n, rp, col, val32 ? NULL : val, val32};
  double *m = f32 ? round32_copy(B, n * (int64_t)bs) : NULL;
  or_ctx c = {&Ain, f32 != 0, 0, NULL, 0, NULL, f32 ? m : B, bs};
  *out = reliable_core(&c, &A64, solver, b, x, tol, maxit, delta);
  free(m);
  return out->status;
}

/* Batched CG with reliable updates: the single-system reliable-update CG
 * above applied to each system of a batch laid out as in or_batch_cg.  val:
 * the systems' FP64 values (replaced residuals); val32: their FP32 values
 * (the recurrences).  Systems spread over the OpenMP threads; each solve is
 * sequential.  iters, updates, relres, status: per system. */
void or_batch_cg_reliable(int32_t count, const int64_t *row_off, const int64_t *nnz_off, const int32_t *rp,
                          const int32_t *col, const double *val, const float *val32, const double *b, double *x,
                          double tol, int32_t maxit, double delta, int32_t *iters, int32_t *updates,
                          double *relres, int32_t *status) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
#endif
  for (int32_t i = 0; i < count; ++i) {
    const int64_t r0 = row_off[i], k0 = nnz_off[i], n = row_off[i + 1] - r0;
    or_op A64 = {n, rp + r0 + i, col + k0, val + k0, NULL};
    or_op A32 = {n, rp + r0 + i, col + k0, NULL, val32 + k0};
    or_ctx c = {&A32, 1, 0, NULL, 0, NULL};
    const or_result res = reliable_core(&c, &A64, OR_SOLVER_CG, b + r0, x + r0, tol, maxit, delta);
    iters[i] = res.iterations;
    updates[i] = res.outer_iterations;
    relres[i] = res.rel_residual;
    status[i] = res.status;
  }
}
