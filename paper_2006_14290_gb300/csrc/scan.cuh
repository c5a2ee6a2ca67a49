// Deterministic device exclusive scan used by planning and format
// conversions (integer only, so the result is exact).
#pragma once

#include "common.cuh"

namespace gko {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* total) {
  __shared__ int64_t warp_tot[kScanThreads / kWarp];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += t;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  int64_t pre = 0, tot = 0;
#pragma unroll
  for (int i = 0; i < kScanThreads / kWarp; ++i) {
    const int64_t t = warp_tot[i];
    if (i < w) pre += t;
    tot += t;
  }
  __syncthreads();
  *total = tot;
  return pre + inc - v;
}

template <typename F>
__global__ void __launch_bounds__(kScanThreads) scan_tile_sums_kernel(F f, int64_t n, int64_t* sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t s = 0;
#pragma unroll
  for (int u = 0; u < kScanItems; ++u)
    if (base + u < n) s += f(base + u);
  int64_t tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// One block: exclusive scan of the m tile sums in place; sums[m] = total.
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(int64_t* sums, int64_t m) {
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < m; b0 += kScanTile) {
    const int64_t base = b0 + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int u = 0; u < kScanItems; ++u) {
      v[u] = (base + u < m) ? sums[base + u] : 0;
      s += v[u];
    }
    int64_t tot;
    int64_t pre = block_exclusive_scan(s, &tot) + carry;
#pragma unroll
    for (int u = 0; u < kScanItems; ++u) {
      if (base + u < m) sums[base + u] = pre;
      pre += v[u];
    }
    carry += tot;
  }
  if (threadIdx.x == 0) sums[m] = carry;
}

template <typename F, typename OutT>
__global__ void __launch_bounds__(kScanThreads)
    scan_tiles_kernel(F f, int64_t n, const int64_t* offs, OutT* out) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int u = 0; u < kScanItems; ++u) {
    v[u] = (base + u < n) ? f(base + u) : 0;
    s += v[u];
  }
  int64_t tot;
  int64_t pre = block_exclusive_scan(s, &tot) + offs[blockIdx.x];
#pragma unroll
  for (int u = 0; u < kScanItems; ++u) {
    if (base + u < n) out[base + u] = (OutT)pre;
    pre += v[u];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = (OutT)offs[gridDim.x];
}

// out[0..n] = exclusive prefix sums of f(0..n-1), out[n] = total.  The total
// is also returned on the host (the call synchronises the stream).
template <typename F, typename OutT>
int exclusive_scan(F f, int64_t n, OutT* out, int64_t* total, cudaStream_t s) {
  const int64_t tiles = n > 0 ? (n + kScanTile - 1) / kScanTile : 1;
  Scratch sums;
  GKO_TRY(sums.get(sizeof(int64_t) * (tiles + 1), s));
  int64_t* d = sums.as<int64_t>();
  scan_tile_sums_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(f, n, d);
  scan_sums_kernel<<<1, kScanThreads, 0, s>>>(d, tiles);
  scan_tiles_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(f, n, d, out);
  GKO_TRY_CUDA(cudaGetLastError());
  GKO_TRY_CUDA(cudaMemcpyAsync(total, d + tiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  return GKO_OK;
}

}  // namespace gko
