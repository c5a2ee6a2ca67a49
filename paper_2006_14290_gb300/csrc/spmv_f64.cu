// SpMV instantiation for double matrix values with double vectors.
#include "spmv_kernels.cuh"

namespace gko {

int spmv_run_f64(const gko_matrix_s* A, const double* x, double* y, double alpha, double beta, cudaStream_t s,
                 void* scratch, const DotSpec* dot, const int* gate) {
  return SpmvImpl<double, double>::run(A, x, y, alpha, beta, s, scratch, dot, gate);
}

}  // namespace gko
