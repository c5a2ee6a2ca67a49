// Deterministic block and grid reductions (FP64) shared by the SpMV,
// BLAS-1 and solver kernels.  No floating-point atomics: blocks publish
// partial sums and the last block to take an integer ticket adds them in
// index order, then runs an optional scalar operation on the totals.
#pragma once

#include "spmv.cuh"

namespace gko {

// Sum of NV values over a block; the totals are valid in thread 0.
template <int THREADS, int NV>
__device__ __forceinline__ void block_sum_n(double (&v)[NV]) {
  __shared__ double red[NV][THREADS / kWarp];
  const int w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    v[k] = subwarp_sum<32>(v[k], 0xffffffffu);
    if ((threadIdx.x & 31) == 0) red[k][w] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < THREADS / kWarp; ++i) s += red[k][i];
      v[k] = s;
    }
  }
  __syncthreads();
}

template <int THREADS>
__device__ __forceinline__ double block_sum(double v) {
  double a[1] = {v};
  block_sum_n<THREADS, 1>(a);
  return a[0];
}

struct NoOp {
  template <int NV>
  __device__ void operator()(const double (&)[NV]) const {}
};

// Store this block's NV partials in `slot`; the block that takes the last of
// `expected` tickets adds all partials in index order and calls op(totals)
// from its thread 0, then re-arms the counter.
template <int THREADS, int NV, typename Op>
__device__ void grid_reduce(double (&v)[NV], double* partials, unsigned* counter, int slot, int expected, Op op) {
  __shared__ int is_last;
  block_sum_n<THREADS, NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[(int64_t)slot * NV + k] = v[k];
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    is_last = (t == (unsigned)expected - 1u);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
#pragma unroll 4
  for (int i = threadIdx.x; i < expected; i += THREADS)
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += __ldcg(partials + (int64_t)i * NV + k);
  block_sum_n<THREADS, NV>(acc);
  if (threadIdx.x == 0) {
    op(acc);
    *counter = 0u;
  }
}

struct StoreOp2 {
  double* result;
  __device__ void operator()(const double (&t)[2]) const {
    result[0] = t[0];
    result[1] = t[1];
  }
};

// Fused dot epilogue of the SpMV kernels: result[0] = w . y, result[1] = y . y.
template <int THREADS>
__device__ __forceinline__ void dot_epilogue2(double wy, double yy, const DotSpec& d, int slot, int expected) {
  double v[2] = {wy, yy};
  grid_reduce<THREADS, 2>(v, d.partials, d.counter, slot, expected, StoreOp2{d.result});
}

// A kernel is gated off when either gate word is nonzero (solver state:
// converged/stopped, or a phase that skips this product).
__device__ __forceinline__ bool gated(const int* g) {
  if (!g) return false;
  return (*(volatile const int*)g | *((volatile const int*)g + 1)) != 0;
}

}  // namespace gko
