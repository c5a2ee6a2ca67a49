// Jacobi preconditioner setup: the inverse diagonal of an FP64 matrix in any
// format (the preconditioner the paper's Section 1 names beside its Krylov
// solvers; M = diag(A), Saad, Iterative Methods for Sparse Linear Systems,
// Sec. 10.2).  The diagonal entries of a row are summed in CSR storage order
// (duplicates add up as in the SpMV); a zero or missing diagonal gives 1, so
// that row is left unscaled.
#include "spmv.cuh"

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

#undef GKO_ROWS

}  // namespace

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
