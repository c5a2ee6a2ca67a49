// SpMV instantiation for float matrix values with float vectors.
#include "spmv_kernels.cuh"

namespace gko {

int spmv_run_f32(const gko_matrix_s* A, const float* x, float* y, double alpha, double beta, cudaStream_t s,
                 void* scratch, const DotSpec* dot, const int* gate) {
  return SpmvImpl<float, float>::run(A, x, y, alpha, beta, s, scratch, dot, gate);
}

}  // namespace gko
