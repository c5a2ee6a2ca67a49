// Jacobi preconditioner setup: the inverse diagonal of an FP64 matrix in any
// format (the preconditioner the paper's Section 1 names beside its Krylov
// solvers; M = diag(A), Saad, Iterative Methods for Sparse Linear Systems,
// Sec. 10.2).  The diagonal entries of a row are summed in CSR storage order
// (duplicates add up as in the SpMV); a zero or missing diagonal gives 1, so
// that row is left unscaled.
#include "precond.cuh"

namespace gko {
namespace {

unsigned grid1d(int64_t work) {
  const int64_t b = (work + 255) / 256;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 65535));
}

#define GKO_ROWS(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__global__ void diag_csr_kernel(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                const double* __restrict__ val, double* __restrict__ d) {
  GKO_ROWS(i, n) {
    double s = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
      if (col[k] == i) s += val[k];
    d[i] = s;
  }
}

// ELL (stride, K) and SELL-P (slices of C rows, sets[]) walk a row's slots
// in storage order.
__global__ void diag_ell_kernel(int64_t n, int32_t K, int64_t stride, const int32_t* __restrict__ col,
                                const double* __restrict__ val, double* __restrict__ d) {
  GKO_ROWS(i, n) {
    double s = 0.0;
    for (int32_t k = 0; k < K; ++k) {
      const int64_t q = (int64_t)k * stride + i;
      if (col[q] == i) s += val[q];
    }
    d[i] = s;
  }
}

__global__ void diag_sellp_kernel(int64_t n, int32_t C, const int32_t* __restrict__ sets,
                                  const int32_t* __restrict__ col, const double* __restrict__ val,
                                  double* __restrict__ d) {
  GKO_ROWS(i, n) {
    const int64_t sl = i / C;
    const int64_t b = sets[sl];
    const int32_t w = sets[sl + 1] - sets[sl];
    double s = 0.0;
    for (int32_t k = 0; k < w; ++k) {
      const int64_t q = (b + k) * C + (i - sl * C);
      if (col[q] == i) s += val[q];
    }
    d[i] = s;
  }
}

// COO (row-sorted): the first diagonal entry of a row adds all of that row's
// diagonal entries, in order, to d[row] (which holds 0, or the ELL part of a
// hybrid matrix).
__global__ void diag_coo_kernel(int64_t nnz, const int32_t* __restrict__ row, const int32_t* __restrict__ col,
                                const double* __restrict__ val, double* __restrict__ d) {
  GKO_ROWS(k, nnz) {
    const int32_t r = row[k];
    if (col[k] != r) continue;
    bool first = true;
    for (int64_t u = k - 1; u >= 0 && row[u] == r; --u)
      if (col[u] == r) {
        first = false;
        break;
      }
    if (!first) continue;
    double s = d[r];
    for (int64_t u = k; u < nnz && row[u] == r; ++u)
      if (col[u] == r) s += val[u];
    d[r] = s;
  }
}

__global__ void invert_kernel(int64_t n, double* __restrict__ d) {
  GKO_ROWS(i, n) d[i] = d[i] != 0.0 ? 1.0 / d[i] : 1.0;
}

__global__ void narrow_kernel(int64_t n, const double* __restrict__ d, float* __restrict__ f) {
  GKO_ROWS(i, n) f[i] = (float)d[i];
}

// Block-Jacobi setup (M = the diagonal blocks of A, Saad Sec. 12.2): one
// warp per block of nb = min(bs, n - base) rows, the augmented [D | I] in
// shared memory (row stride 2 bs + 1 doubles), Gauss-Jordan elimination with partial
// pivoting: the first row of largest magnitude in the pivot column, the
// pivot row multiplied by the reciprocal of the pivot (one division per
// step), then every other row r takes row_r - m_r row_k, products and
// differences rounded separately, never fused.  The pivot search and the
// row swap run over lanes = rows / columns; the elimination spreads the
// entries still read later (columns k+1 .. 2 nb - 1 of every row) over the
// 32 lanes, with the multipliers m_r (the pivot column before the step)
// staged in shared memory first, so each entry of the inverse gets exactly
// the operations of the sequential elimination.  A block whose
// pivot column is all zero at some step is left unscaled (identity rows)
// and counted in *singular.
__global__ void bj_setup_kernel(int64_t n, int bs, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                const double* __restrict__ val, double* __restrict__ B,
                                unsigned long long* singular) {
  extern __shared__ double bj_smem[];
  const int lane = threadIdx.x & 31;
  const int wpc = blockDim.x >> 5;
  const int ST = 2 * bs + 1;
  double* M = bj_smem + (size_t)(threadIdx.x >> 5) * (bs * ST + bs);
  double* mk = M + bs * ST;  // multipliers of the current step
  const int64_t blocks = (n + bs - 1) / bs;
  for (int64_t blk = (int64_t)blockIdx.x * wpc + (threadIdx.x >> 5); blk < blocks; blk += (int64_t)gridDim.x * wpc) {
    const int64_t base = blk * bs;
    const int nb = (int)(n - base < bs ? n - base : bs);
    const int w = 2 * nb;
    for (int e = lane; e < nb * ST; e += 32) M[e] = 0.0;
    __syncwarp();
    if (lane < nb) {
      M[lane * ST + nb + lane] = 1.0;
      for (int32_t k = rp[base + lane]; k < rp[base + lane + 1]; ++k) {
        const int64_t c = (int64_t)col[k] - base;
        if (c >= 0 && c < nb) M[lane * ST + c] += val[k];
      }
    }
    __syncwarp();
    bool ok = true;
    for (int k = 0; k < nb; ++k) {
      // Pivot search on the magnitudes' bit patterns: for non-negative
      // doubles (not NaN) the unsigned 64-bit order is the numeric order, so
      // the arg-max runs on the integer pipe instead of GB300's narrow FP64
      // pipe (FP64 compares in this butterfly were most of the setup's FP64
      // work).  Lanes outside rows k .. nb-1 offer 0.
      constexpr unsigned long long kMag = ~(1ull << 63);
      unsigned long long a =
          (lane >= k && lane < nb) ? ((unsigned long long)__double_as_longlong(M[lane * ST + k]) & kMag) : 0ull;
      int idx = lane;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long oa = __shfl_xor_sync(0xffffffffu, a, off);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, off);
        if (oa > a || (oa == a && oi < idx)) {
          a = oa;
          idx = oi;
        }
      }
      // the butterfly leaves every lane with the same pivot; lane 0's copy
      // and a vote keep the control flow warp-uniform
      a = __shfl_sync(0xffffffffu, a, 0);
      idx = __shfl_sync(0xffffffffu, idx, 0);
      if (__any_sync(0xffffffffu, a == 0ull)) {
        ok = false;
        break;
      }
      if (idx != k)
        for (int c = lane; c < w; c += 32) {
          const double t = M[k * ST + c];
          M[k * ST + c] = M[idx * ST + c];
          M[idx * ST + c] = t;
        }
      __syncwarp();
      // one division per step, by lane 0 (FP64 division is a long sequence
      // on GB300's narrow FP64 pipe)
      double inv = 0.0;
      if (lane == 0) inv = 1.0 / M[k * ST + k];
      inv = __shfl_sync(0xffffffffu, inv, 0);
      // Columns 0..k of the left half are never read again after this step
      // (later pivot searches and multipliers read columns above k), so only
      // columns k+1 .. 2nb-1 are scaled and eliminated: the right half, the
      // inverse, gets exactly the sequential elimination's operations.
      const int c0 = k + 1, wc = w - c0;
      for (int c = c0 + lane; c < w; c += 32) M[k * ST + c] = __dmul_rn(M[k * ST + c], inv);
      if (lane < nb) mk[lane] = M[lane * ST + k];
      __syncwarp();
      for (int e = lane; e < nb * wc; e += 32) {
        const int r = e / wc, c = c0 + (e - r * wc);
        if (r != k) M[r * ST + c] = __dsub_rn(M[r * ST + c], __dmul_rn(mk[r], M[k * ST + c]));
      }
      __syncwarp();
    }
    for (int r = 0; r < nb; ++r)
      for (int j = lane; j < bs; j += 32)
        B[(base + r) * bs + j] = j < nb ? (ok ? M[r * ST + nb + j] : (r == j ? 1.0 : 0.0)) : 0.0;
    if (!ok && lane == 0 && singular) atomicAdd(singular, 1ull);
    __syncwarp();
  }
}

#undef GKO_ROWS

}  // namespace

int block_jacobi_inverse(const gko_matrix_s* A, int bs, double* B, unsigned long long* singular, cudaStream_t s) {
  if (A->dtype != GKO_F64 || A->fmt != GKO_CSR)
    return fail(GKO_NOT_SUPPORTED, "the block-Jacobi setup reads an FP64 CSR matrix");
  if (bs < 1 || bs > kBlockJacobiMax) return fail(GKO_INVALID_ARG, "block-Jacobi block size must lie in 1..32");
  const int64_t n = A->n_rows;
  if (n == 0) return GKO_OK;
  const int wpc = bs > 16 ? 2 : 4;  // warps per block: at most 34 KB of shared memory
  const size_t smem = sizeof(double) * (size_t)wpc * (bs * (2 * bs + 1) + bs);
  const int64_t blocks = (n + bs - 1) / bs;
  const int64_t g = std::max<int64_t>(1, std::min<int64_t>((blocks + wpc - 1) / wpc, (int64_t)sm_count() * 32));
  bj_setup_kernel<<<(unsigned)g, 32 * wpc, smem, s>>>(n, bs, ptr<int32_t>(A->row_ptr), ptr<int32_t>(A->col),
                                                      ptr<double>(A->val), B, singular);
  GKO_TRY_CUDA(cudaGetLastError());
  return GKO_OK;
}

int jacobi_inverse(const gko_matrix_s* A, double* d, cudaStream_t s) {
  if (A->dtype != GKO_F64) return fail(GKO_INVALID_ARG, "the Jacobi setup reads the FP64 matrix");
  const int64_t n = A->n_rows;
  if (n == 0) return GKO_OK;
  const unsigned g = grid1d(n);
  switch (A->fmt) {
    case GKO_CSR:
      diag_csr_kernel<<<g, 256, 0, s>>>(n, ptr<int32_t>(A->row_ptr), ptr<int32_t>(A->col), ptr<double>(A->val), d);
      break;
    case GKO_ELL:
    case GKO_HYBRID:
      diag_ell_kernel<<<g, 256, 0, s>>>(n, A->K, A->stride, ptr<int32_t>(A->ell_col), ptr<double>(A->ell_val), d);
      break;
    case GKO_SELLP:
      diag_sellp_kernel<<<g, 256, 0, s>>>(n, A->slice, ptr<int32_t>(A->sellp_sets), ptr<int32_t>(A->sellp_col),
                                          ptr<double>(A->sellp_val), d);
      break;
    case GKO_COO:
      GKO_TRY_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * n, s));
      break;
  }
  if ((A->fmt == GKO_COO || A->fmt == GKO_HYBRID) && A->coo_nnz > 0)
    diag_coo_kernel<<<grid1d(A->coo_nnz), 256, 0, s>>>(A->coo_nnz, ptr<int32_t>(A->coo_row), ptr<int32_t>(A->coo_col),
                                                       ptr<double>(A->coo_val), d);
  invert_kernel<<<g, 256, 0, s>>>(n, d);
  GKO_TRY_CUDA(cudaGetLastError());
  return GKO_OK;
}

int narrow_to_f32(const double* d, float* f, int64_t n, cudaStream_t s) {
  if (n == 0) return GKO_OK;
  narrow_kernel<<<grid1d(n), 256, 0, s>>>(n, d, f);
  GKO_TRY_CUDA(cudaGetLastError());
  return GKO_OK;
}

}  // namespace gko

extern "C" {

int gko_block_jacobi_inverse(gko_matrix A, int32_t block_size, double* B, int64_t* singular, void* stream) {
  if (!A) return gko::fail(GKO_INVALID_ARG, "null matrix");
  if (A->n_rows != A->n_cols) return gko::fail(GKO_INVALID_ARG, "block-Jacobi needs a square matrix");
  if (A->n_rows > 0 && !B) return gko::fail(GKO_INVALID_ARG, "null B");
  cudaStream_t s = (cudaStream_t)stream;
  gko::Scratch cnt;
  unsigned long long* dc = nullptr;
  if (singular) {
    GKO_TRY(cnt.get(sizeof(unsigned long long), s));
    dc = cnt.as<unsigned long long>();
    GKO_TRY_CUDA(cudaMemsetAsync(dc, 0, sizeof(unsigned long long), s));
  }
  GKO_TRY(gko::block_jacobi_inverse(A, block_size, B, dc, s));
  if (singular) {
    unsigned long long h = 0;
    GKO_TRY_CUDA(cudaMemcpyAsync(&h, dc, sizeof h, cudaMemcpyDeviceToHost, s));
    GKO_TRY_CUDA(cudaStreamSynchronize(s));
    *singular = (int64_t)h;
  }
  return GKO_OK;
}

}  // extern "C"
