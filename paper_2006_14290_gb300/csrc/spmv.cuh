// SpMV kernels y = alpha*A*x + beta*y for the formats the paper lists
// (Section 1: Coo, Csr, Ell, Hybrid) and the internal dispatch used by the
// C ABI and the Krylov solvers.  All kernels are deterministic: a fixed
// launch shape and fixed summation order give bit-identical results on
// every call, with no floating-point atomics.
#pragma once

#include "common.cuh"

namespace gko {

// Fused dot epilogue: result[0] = sum_i w[i] * y[i] and result[1] =
// sum_i y[i]^2, in FP64 over the rows the SpMV writes.  Blocks store partial
// sums; the last block to arrive (integer ticket) adds them in index order,
// so the values are deterministic.
struct DotSpec {
  const void* w = nullptr;  // same element type as y
  double* partials = nullptr;  // 2 * kDotSlots doubles
  unsigned* counter = nullptr;  // zero on entry; the last block resets it
  double* result = nullptr;     // 2 doubles
  int want_yy = 1;              // 0: skip y.y (result[1] = 0)
};
constexpr int kDotSlots = 4096;  // blocks a fused reduction may use

// Scratch bytes one SpMV of A needs (long-row partials or COO carries).
size_t spmv_scratch_bytes(const gko_matrix_s* A);
// Whether spmv_run can fuse the dot epilogue for this format.
bool spmv_fuses_dot(const gko_matrix_s* A);

// x, y: device vectors (double for F64 matrices, float otherwise).
// gate (nullable): two device ints; every kernel returns at once when either
// is nonzero (used by the solvers to turn finished iterations into no-ops).
int spmv_run(const gko_matrix_s* A, const void* x, void* y, double alpha, double beta, cudaStream_t s,
             void* scratch, const DotSpec* dot, const int* gate = nullptr);

// Per value type entry points (one translation unit each).
int spmv_run_f64(const gko_matrix_s* A, const double* x, double* y, double alpha, double beta, cudaStream_t s,
                 void* scratch, const DotSpec* dot, const int* gate);
int spmv_run_f32(const gko_matrix_s* A, const float* x, float* y, double alpha, double beta, cudaStream_t s,
                 void* scratch, const DotSpec* dot, const int* gate);
int spmv_run_bf16(const gko_matrix_s* A, const float* x, float* y, double alpha, double beta, cudaStream_t s,
                  void* scratch, const DotSpec* dot, const int* gate);

// Jacobi preconditioner: d = inverse diagonal of the FP64 matrix A (any
// format; zero diagonal -> 1), and its FP32 rounding for inner solves.
int jacobi_inverse(const gko_matrix_s* A, double* d, cudaStream_t s);
int narrow_to_f32(const double* d, float* f, int64_t n, cudaStream_t s);

constexpr int kCooThreads = 128;
constexpr int kCooItems = 8;
constexpr int kCooTile = kCooThreads * kCooItems;

}  // namespace gko
