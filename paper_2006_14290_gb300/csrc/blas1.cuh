// Deterministic vector kernels (the BLAS-1 part of the Krylov solvers):
// dot / nrm2 with FP64 accumulation, axpy, fused multi-dot and fused
// multi-axpy + norm (the Gram-Schmidt passes of GMRES).
#pragma once

#include "reduce.cuh"

namespace gko {

// Workspace of a grid reduction: kDotSlots partials and a zeroed counter.
struct RedWs {
  double* partials;
  unsigned* counter;
};

int reduce_grid(int64_t n);

// *result (device) = x . y, FP64 accumulation; T = double or float.
template <typename T>
int dot_launch(int64_t n, const T* x, const T* y, double* result, RedWs ws, cudaStream_t s);
// y = a*x + y
int axpy_launch(int64_t n, double a, const double* x, double* y, cudaStream_t s);
// h[j] = V_j . w for j < k (h on the device); partials: k * kMultiSlots doubles.
constexpr int kMultiSlots = 256;
template <typename T>
int multi_dot_launch(int64_t n, int32_t k, const T* V, int64_t ldv, const T* w, double* h, double* partials,
                     cudaStream_t s);
// y -= sum_j h[j] V_j, then *result = ||y||^2 (device, FP64).
template <typename T>
int multi_axpy_norm_launch(int64_t n, int32_t k, const double* h, const T* V, int64_t ldv, T* y, double* result,
                           RedWs ws, cudaStream_t s);

}  // namespace gko
