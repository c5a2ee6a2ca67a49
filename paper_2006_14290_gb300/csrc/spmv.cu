// SpMV dispatch over value types and the gko_spmv entry point.
#include "spmv.cuh"

namespace gko {

size_t spmv_scratch_bytes(const gko_matrix_s* A) {
  const size_t at = A->dtype == GKO_F64 ? 8 : 4;
  switch (A->fmt) {
    case GKO_CSR:
      if (A->plan.kind == 2) return at * 2 * (size_t)((A->n_rows + A->nnz + 2047) / 2048 + 1);
      return at * (size_t)A->plan.n_chunks;
    case GKO_ELL:
    case GKO_SELLP:
      return 0;
    case GKO_COO:
      if (A->plan.kind == 1) return 0;
      return at * 2 * (size_t)((A->coo_nnz + kCooTile - 1) / kCooTile);
    case GKO_HYBRID:
      return at * 2 * (size_t)((A->coo_nnz + kCooTile - 1) / kCooTile);
  }
  return 0;
}

bool spmv_fuses_dot(const gko_matrix_s* A) {
  return (A->fmt == GKO_CSR && A->plan.kind != 2) || A->fmt == GKO_ELL || A->fmt == GKO_SELLP ||
         (A->fmt == GKO_COO && A->plan.kind == 1 && A->coo_nnz > 0);
}

int spmv_run(const gko_matrix_s* A, const void* x, void* y, double alpha, double beta, cudaStream_t s, void* scratch,
             const DotSpec* dot, const int* gate) {
  switch (A->dtype) {
    case GKO_F64:
      return spmv_run_f64(A, static_cast<const double*>(x), static_cast<double*>(y), alpha, beta, s, scratch, dot, gate);
    case GKO_F32:
      return spmv_run_f32(A, static_cast<const float*>(x), static_cast<float*>(y), alpha, beta, s, scratch, dot, gate);
    case GKO_BF16:
      return spmv_run_bf16(A, static_cast<const float*>(x), static_cast<float*>(y), alpha, beta, s, scratch, dot, gate);
  }
  return fail(GKO_INVALID_ARG, "bad dtype");
}

}  // namespace gko

using namespace gko;

extern "C" int gko_spmv(const double* alpha, gko_matrix A, const void* x, const double* beta, void* y,
                        gko_dtype vec_dtype, void* stream) {
  if (!A || !alpha || !beta) return fail(GKO_INVALID_ARG, "null matrix or scalar");
  if (A->n_rows > 0 && !y) return fail(GKO_INVALID_ARG, "null y");
  if (A->n_cols > 0 && A->nnz > 0 && !x) return fail(GKO_INVALID_ARG, "null x");
  const gko_dtype need = A->dtype == GKO_F64 ? GKO_F64 : GKO_F32;
  if (vec_dtype != need)
    return fail(GKO_INVALID_ARG, "vector dtype must be F64 for F64 matrices and F32 for F32/BF16 matrices");
  if (A->n_rows == 0) return GKO_OK;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scratch;
  const size_t sb = spmv_scratch_bytes(A);
  if (sb) GKO_TRY(scratch.get(sb, s));
  return spmv_run(A, x, y, *alpha, *beta, s, scratch.data(), nullptr);
}

// SpMV on host vectors: stream-ordered copies around gko_spmv (see gko.h).
extern "C" int gko_spmv_host(const double* alpha, gko_matrix A, const void* x_host, const double* beta,
                             void* y_host, gko_dtype vec_dtype, void* x_dev, void* y_dev, void* stream) {
  if (!A || !alpha || !beta) return fail(GKO_INVALID_ARG, "null matrix or scalar");
  if (A->n_rows > 0 && (!y_host || !y_dev)) return fail(GKO_INVALID_ARG, "null y");
  if (A->n_cols > 0 && (!x_host || !x_dev)) return fail(GKO_INVALID_ARG, "null x");
  const size_t es = vec_dtype == GKO_F64 ? sizeof(double) : sizeof(float);
  cudaStream_t s = (cudaStream_t)stream;
  if (A->n_cols > 0)
    GKO_TRY_CUDA(cudaMemcpyAsync(x_dev, x_host, es * (size_t)A->n_cols, cudaMemcpyHostToDevice, s));
  if (A->n_rows > 0 && *beta != 0.0)
    GKO_TRY_CUDA(cudaMemcpyAsync(y_dev, y_host, es * (size_t)A->n_rows, cudaMemcpyHostToDevice, s));
  GKO_TRY(gko_spmv(alpha, A, x_dev, beta, y_dev, vec_dtype, stream));
  if (A->n_rows > 0)
    GKO_TRY_CUDA(cudaMemcpyAsync(y_host, y_dev, es * (size_t)A->n_rows, cudaMemcpyDeviceToHost, s));
  return GKO_OK;
}

