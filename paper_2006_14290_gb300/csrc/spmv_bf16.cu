// SpMV instantiation for __nv_bfloat16 matrix values with float vectors.
#include "spmv_kernels.cuh"

namespace gko {

int spmv_run_bf16(const gko_matrix_s* A, const float* x, float* y, double alpha, double beta, cudaStream_t s,
                  void* scratch, const DotSpec* dot, const int* gate) {
  return SpmvImpl<__nv_bfloat16, float>::run(A, x, y, alpha, beta, s, scratch, dot, gate);
}

}  // namespace gko
