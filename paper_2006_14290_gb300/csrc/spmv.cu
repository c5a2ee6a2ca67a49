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
