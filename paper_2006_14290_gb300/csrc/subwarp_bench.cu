// Subwarp reduction microbenchmark (paper, Section 3.3: the reduce listing
// and the 2000 - 1000 inner-loop difference method).  A block of 256
// threads reads one value per thread, runs `inner_loops` butterfly
// reductions over subwarps of S lanes and writes the result back, so the
// time of 1000 reductions is t(2000 loops) - t(1000 loops) with launch and
// memory costs cancelled.  Three implementations of the same butterfly:
//   0  the library's subwarp primitive (subwarp_mask + masked xor shuffle of
//      width S), the one the SpMV and Krylov kernels use;
//   1  CUDA cooperative groups (tiled_partition<S>(this_thread_block())),
//      the interface the paper's cross-platform layer mirrors;
//   2  the plain full-warp xor shuffle with width S (the "legacy" intrinsic).
#include <cooperative_groups.h>

#include "common.cuh"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace gko {
namespace {

constexpr int kBenchThreads = 256;

template <int S, int IMPL, typename T>
__device__ __forceinline__ T butterfly(T v) {
  if (IMPL == 0) return subwarp_sum<S>(v, subwarp_mask<S>());
  if (IMPL == 1) {
    auto group = cg::tiled_partition<S>(cg::this_thread_block());
#pragma unroll
    for (int bitmask = 1; bitmask < S; bitmask <<= 1) v = v + group.shfl_xor(v, bitmask);
    return v;
  }
#pragma unroll
  for (int bitmask = 1; bitmask < S; bitmask <<= 1) v = v + __shfl_xor_sync(0xffffffffu, v, bitmask, S);
  return v;
}

template <int S, int IMPL, typename T>
__global__ void __launch_bounds__(kBenchThreads) subwarp_reduce_kernel(T* __restrict__ data, int inner_loops) {
  const int64_t i = (int64_t)blockIdx.x * kBenchThreads + threadIdx.x;
  T v = data[i];
  for (int it = 0; it < inner_loops; ++it) v = butterfly<S, IMPL>(v);
  data[i] = v;
}

template <typename T, int IMPL>
int launch_impl(int32_t S, T* data, int64_t n, int32_t loops, cudaStream_t s) {
  const unsigned blocks = (unsigned)(n / kBenchThreads);
  switch (S) {
    case 1: subwarp_reduce_kernel<1, IMPL><<<blocks, kBenchThreads, 0, s>>>(data, loops); break;
    case 2: subwarp_reduce_kernel<2, IMPL><<<blocks, kBenchThreads, 0, s>>>(data, loops); break;
    case 4: subwarp_reduce_kernel<4, IMPL><<<blocks, kBenchThreads, 0, s>>>(data, loops); break;
    case 8: subwarp_reduce_kernel<8, IMPL><<<blocks, kBenchThreads, 0, s>>>(data, loops); break;
    case 16: subwarp_reduce_kernel<16, IMPL><<<blocks, kBenchThreads, 0, s>>>(data, loops); break;
    case 32: subwarp_reduce_kernel<32, IMPL><<<blocks, kBenchThreads, 0, s>>>(data, loops); break;
    default: return fail(GKO_INVALID_ARG, "subwarp must be 1, 2, 4, 8, 16 or 32");
  }
  GKO_TRY_CUDA(cudaGetLastError());
  return GKO_OK;
}

template <typename T>
int launch_typed(int32_t S, int32_t impl, T* data, int64_t n, int32_t loops, cudaStream_t s) {
  if (impl == 0) return launch_impl<T, 0>(S, data, n, loops, s);
  if (impl == 1) return launch_impl<T, 1>(S, data, n, loops, s);
  return launch_impl<T, 2>(S, data, n, loops, s);
}

// FMA throughput probe: every thread runs 8 independent chains
// v = fma(v, a, b) in registers (a = 1 - 2^-10, b = 2^-10, so each chain
// tends to 1 and stays finite) and stores the sum of its chains.  No memory
// traffic inside the loop, so the difference of two loop counts over the
// difference of their times is the FMA pipe's rate; used to state FP64
// fractions next to the HBM fractions (GB300's FP64 pipe co-limits the FP64
// kernels).
template <typename T>
__global__ void __launch_bounds__(kBenchThreads) fma_chain_kernel(T* __restrict__ data, int loops) {
  const int64_t i = (int64_t)blockIdx.x * kBenchThreads + threadIdx.x;
  const T a = (T)0.9990234375, b = (T)0.0009765625;
  T v[8];
  const T x0 = data[i];
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c] = x0 + (T)c * (T)0.125;
  for (int it = 0; it < loops; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = fma(v[c], a, b);
  }
  T sum = (T)0;
#pragma unroll
  for (int c = 0; c < 8; ++c) sum += v[c];
  data[i] = sum;
}

// Random-gather throughput probe: every thread keeps 8 independent index
// streams (a 32-bit linear congruential step each, indices = the state's
// top bits masked to the power-of-two vector length) and gathers one
// element per stream per loop from x, folding the element's bits into an
// integer xor so no floating-point pipe is involved; the load addresses
// never depend on loaded data, so every gather of a loop can be in flight.
// This is the access pattern of an SpMV whose columns are uniformly random
// (the power-law matrices): one 8- or 4-byte element per L2 sector.
constexpr uint32_t kLcgA = 1664525u, kLcgC = 1013904223u;
template <typename U>
__global__ void __launch_bounds__(kBenchThreads) gather_kernel(const U* __restrict__ x, uint32_t mask, int shift,
                                                               U* __restrict__ out, int loops) {
  const int64_t i = (int64_t)blockIdx.x * kBenchThreads + threadIdx.x;
  uint32_t st[8];
  U acc = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) st[c] = (uint32_t)i * 8u + (uint32_t)c;
  for (int it = 0; it < loops; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      st[c] = st[c] * kLcgA + kLcgC;
      acc ^= __ldcg(x + ((st[c] >> shift) & mask));
    }
  }
  out[i] = acc;
}

// Failure-detection check of the bounded waits: one warp waits on an
// mbarrier that nothing ever completes, through the same bounded wait the
// bulk-copy pipelines use, but with a caller-given cycle limit.  The wait
// gives up, records GKO_TIMEOUT in the device error word and the kernel
// returns normally; no copy is in flight, so the block may leave.
__global__ void bounded_wait_kernel(long long limit, int* err, int* out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  const bool ok = mbar_wait_for(&bar, 0u, err, limit);
  if (threadIdx.x == 0) *out = ok ? 0 : 1;
}

}  // namespace
}  // namespace gko

using namespace gko;

extern "C" int gko_diag_bounded_wait(int64_t cycles, int32_t* timed_out, void* stream) {
  if (!timed_out || cycles <= 0 || cycles > kWaitCycles)
    return fail(GKO_INVALID_ARG, "cycles must be in 1 .. 2^32 and timed_out non-null");
  cudaStream_t s = (cudaStream_t)stream;
  int* err = device_error_word();
  if (!err) return fail(GKO_CUDA_ERROR, "device error word unavailable");
  Scratch sc;
  GKO_TRY(sc.get(sizeof(int), s));
  bounded_wait_kernel<<<1, 32, 0, s>>>((long long)cycles, err, sc.as<int>());
  GKO_TRY_CUDA(cudaGetLastError());
  int v = 0;
  GKO_TRY_CUDA(cudaMemcpyAsync(&v, sc.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, s));
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  *timed_out = v;
  return GKO_OK;
}

extern "C" int gko_bench_subwarp_reduce(int32_t subwarp, int32_t impl, gko_dtype dtype, int32_t inner_loops,
                                        void* data, int64_t n, void* stream) {
  if (!data || n <= 0 || n % kBenchThreads != 0 || n / kBenchThreads > INT32_MAX || inner_loops < 0 || impl < 0 ||
      impl > 2)
    return fail(GKO_INVALID_ARG, "bad subwarp benchmark arguments (n a positive multiple of 256, impl 0..2)");
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == GKO_F64) return launch_typed(subwarp, impl, static_cast<double*>(data), n, inner_loops, s);
  if (dtype == GKO_F32) return launch_typed(subwarp, impl, static_cast<float*>(data), n, inner_loops, s);
  return fail(GKO_INVALID_ARG, "dtype must be F64 or F32");
}

extern "C" int gko_bench_gather(gko_dtype dtype, int32_t inner_loops, const void* x, int32_t log2_len, void* out,
                                int64_t n, void* stream) {
  if (!x || !out || n <= 0 || n % kBenchThreads != 0 || n / kBenchThreads > INT32_MAX || inner_loops < 0 ||
      log2_len < 1 || log2_len > 30 || (n * 8) >> 32 != 0)
    return fail(GKO_INVALID_ARG, "bad gather benchmark arguments (n a positive multiple of 256, log2_len 1..30)");
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned blocks = (unsigned)(n / kBenchThreads);
  const uint32_t mask = (uint32_t)((1ull << log2_len) - 1);
  const int shift = 32 - log2_len;
  if (dtype == GKO_F64) {
    gather_kernel<unsigned long long><<<blocks, kBenchThreads, 0, s>>>(
        static_cast<const unsigned long long*>(x), mask, shift, static_cast<unsigned long long*>(out), inner_loops);
  } else if (dtype == GKO_F32) {
    gather_kernel<unsigned><<<blocks, kBenchThreads, 0, s>>>(static_cast<const unsigned*>(x), mask, shift,
                                                             static_cast<unsigned*>(out), inner_loops);
  } else {
    return fail(GKO_INVALID_ARG, "dtype must be F64 or F32");
  }
  GKO_TRY_CUDA(cudaGetLastError());
  return GKO_OK;
}

extern "C" int gko_bench_fma(gko_dtype dtype, int32_t inner_loops, void* data, int64_t n, void* stream) {
  if (!data || n <= 0 || n % kBenchThreads != 0 || n / kBenchThreads > INT32_MAX || inner_loops < 0)
    return fail(GKO_INVALID_ARG, "bad FMA benchmark arguments (n a positive multiple of 256)");
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned blocks = (unsigned)(n / kBenchThreads);
  if (dtype == GKO_F64) {
    fma_chain_kernel<double><<<blocks, kBenchThreads, 0, s>>>(static_cast<double*>(data), inner_loops);
  } else if (dtype == GKO_F32) {
    fma_chain_kernel<float><<<blocks, kBenchThreads, 0, s>>>(static_cast<float*>(data), inner_loops);
  } else {
    return fail(GKO_INVALID_ARG, "dtype must be F64 or F32");
  }
  GKO_TRY_CUDA(cudaGetLastError());
  return GKO_OK;
}
