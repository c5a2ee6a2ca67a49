// COO SpMV that allocates nothing: the same tiled segmented-reduction
// kernels as gko_spmv on a COO handle, with their per-tile carry scratch in
// a fixed file-scope device array instead of the stream-ordered pool.
//
// For callers that cannot allocate device memory when they multiply: code
// whose device memory is entirely owned by another allocator (a framework's
// caching allocator or a fixed arena sized at start-up), or latency-critical
// loops where an allocation, with its possible implicit synchronisation, is
// not acceptable.  They create the COO handle once beforehand; this call then
// reads the handle, x and y and touches no allocator.
#include <stdio.h>

#include <mutex>

#include "spmv_kernels.cuh"

namespace gko {

constexpr int64_t kNoAllocMaxNnz = (int64_t)1 << 27;  // 134,217,728 entries
constexpr int64_t kNoAllocMaxTiles = kNoAllocMaxNnz / kCooTile;

// Two FP64 carries per tile (2 MiB).  CUDA loads this file's device code,
// and the array with it, lazily: on a device's first call (or first symbol
// lookup); from then on that device holds the array until the process exits.
static __device__ __align__(256) double g_noalloc_carry[2 * kNoAllocMaxTiles];

static std::mutex g_noalloc_mu;
static double* g_noalloc_addr[64] = {nullptr};

// Device address of the carry array for the current device, looked up once
// per device with that device current (host code may not use the symbol's
// host-side name as a device pointer).
static int noalloc_scratch(double** out) {
  int dev = 0;
  GKO_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(GKO_NOT_SUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_carry);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(carry scratch)");
    g_noalloc_addr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_addr[dev];
  return GKO_OK;
}

}  // namespace gko

using namespace gko;

extern "C" int gko_spmv_coo_noalloc(const double* alpha, gko_matrix A, const double* x, const double* beta,
                                    double* y, void* stream) {
  if (!A || !alpha || !beta) return fail(GKO_INVALID_ARG, "null matrix or scalar");
  if (A->fmt != GKO_COO || A->dtype != GKO_F64) return fail(GKO_INVALID_ARG, "needs an F64 COO handle");
  if (A->coo_nnz > kNoAllocMaxNnz) {
    char msg[160];
    snprintf(msg, sizeof msg, "COO has %lld entries; the allocation-free SpMV supports at most %lld",
             (long long)A->coo_nnz, (long long)kNoAllocMaxNnz);
    return fail(GKO_INVALID_ARG, msg);
  }
  if (A->n_rows > 0 && !y) return fail(GKO_INVALID_ARG, "null y");
  if (A->coo_nnz > 0 && !x) return fail(GKO_INVALID_ARG, "null x");
  if (A->n_rows == 0) return GKO_OK;
  double* carry = nullptr;
  GKO_TRY(noalloc_scratch(&carry));
  cudaStream_t s = (cudaStream_t)stream;
  const double a = *alpha, b = *beta;
  const int64_t nnz = A->coo_nnz;
  if (nnz == 0) {
    const int64_t g = std::max<int64_t>(1, std::min<int64_t>((A->n_rows + 255) / 256, 4096));
    scale_kernel<double, double><<<(unsigned)g, 256, 0, s>>>(A->n_rows, y, b, nullptr);
    GKO_TRY_CUDA(cudaGetLastError());
    return GKO_OK;
  }
  // Every carry slot the fix-up reads is written earlier in the same call, so
  // nothing needs clearing; calls that overlap on the GPU share the array
  // and race.
  CooArgs<double, double> args{A->n_rows, A->n_cols, nnz, ptr<int32_t>(A->coo_row), ptr<int32_t>(A->coo_col),
                               ptr<double>(A->coo_val), x, y, a, b, a == 1.0 && b == 0.0};
  coo_launch<double, double, false>(args, carry, nullptr, s);
  GKO_TRY_CUDA(cudaGetLastError());
  return GKO_OK;
}
