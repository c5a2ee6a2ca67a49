// Library runtime: error reporting, the device-memory budget, budgeted
// allocations and the stream-ordered scratch pool.
#include <stdio.h>

#include "common.cuh"

namespace gko {

static thread_local std::string g_err;

int fail(int status, const std::string& msg) {
  g_err = msg;
  return status;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // allocation failures are not sticky; clear them
    return GKO_OUT_OF_MEMORY;
  }
  return GKO_CUDA_ERROR;
}

void clear_error() { g_err.clear(); }

bool& pdl_launches() {
  static thread_local bool on = false;
  return on;
}

// ------------------------------------------------------------- budget ----

static std::atomic<int64_t> g_budget{0};
static std::atomic<int64_t> g_in_use{0};

int budget_reserve(size_t bytes) {
  const int64_t b = g_budget.load();
  const int64_t cur = g_in_use.fetch_add((int64_t)bytes) + (int64_t)bytes;
  if (b > 0 && cur > b) {
    g_in_use.fetch_sub((int64_t)bytes);
    char msg[160];
    snprintf(msg, sizeof msg, "allocation of %zu bytes exceeds the memory budget (%lld of %lld in use)",
             bytes, (long long)(cur - (int64_t)bytes), (long long)b);
    return fail(GKO_BUDGET_EXCEEDED, msg);
  }
  return GKO_OK;
}

void budget_release(size_t bytes) { g_in_use.fetch_sub((int64_t)bytes); }

DeviceBuffer::~DeviceBuffer() {
  if (ptr) {
    cudaFree(ptr);
    budget_release(bytes);
  }
}

int alloc(size_t bytes, Buf* out) {
  // every buffer is a valid, 256-byte aligned pointer with at least 128 bytes
  // of slack past the requested end, so bulk copies of a tail rounded up to
  // 16-byte granules stay inside the allocation
  bytes = (bytes + 128 + 255) / 256 * 256;
  GKO_TRY(budget_reserve(bytes));
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    budget_release(bytes);
    return cuda_fail(e, "cudaMalloc");
  }
  auto b = std::make_shared<DeviceBuffer>();
  b->ptr = p;
  b->bytes = bytes;
  *out = std::move(b);
  return GKO_OK;
}

// ------------------------------------------------------------ scratch ----

static std::mutex g_pool_mu;
static std::map<int, cudaMemPool_t> g_pools;

static int device_pool(cudaMemPool_t* out) {
  int dev = 0;
  GKO_TRY_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) {
    *out = it->second;
    return GKO_OK;
  }
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool;
  GKO_TRY_CUDA(cudaMemPoolCreate(&pool, &props));
  uint64_t keep = UINT64_MAX;  // keep freed blocks for reuse within the process
  GKO_TRY_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
  g_pools[dev] = pool;
  *out = pool;
  return GKO_OK;
}

int Scratch::get(size_t bytes, cudaStream_t s) {
  if (bytes < 256) bytes = 256;
  cudaMemPool_t pool;
  GKO_TRY(device_pool(&pool));
  GKO_TRY(budget_reserve(bytes));
  cudaError_t e = cudaMallocFromPoolAsync(&p_, bytes, pool, s);
  if (e != cudaSuccess) {
    budget_release(bytes);
    p_ = nullptr;
    return cuda_fail(e, "cudaMallocFromPoolAsync");
  }
  bytes_ = bytes;
  s_ = s;
  return GKO_OK;
}

Scratch::~Scratch() {
  if (p_) {
    cudaFreeAsync(p_, s_);
    budget_release(bytes_);
  }
}

// Device error word: kernels OR in (1 << status) when a bounded wait gives up.
__device__ int g_device_error;

int* device_error_word() {
  static int* cached[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!cached[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_error) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    cached[dev] = static_cast<int*>(p);
  }
  return cached[dev];
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

size_t dtype_size(gko_dtype t) {
  switch (t) {
    case GKO_F64: return 8;
    case GKO_F32: return 4;
    case GKO_BF16: return 2;
  }
  return 0;
}

}  // namespace gko

extern "C" {

const char* gko_last_error(void) { return gko::g_err.c_str(); }

const char* gko_status_string(int s) {
  switch (s) {
    case GKO_OK: return "ok";
    case GKO_INVALID_ARG: return "invalid argument";
    case GKO_OUT_OF_MEMORY: return "out of device memory";
    case GKO_FORMAT_UNSUITABLE: return "format unsuitable (padding limit)";
    case GKO_NOT_CONVERGED: return "not converged";
    case GKO_BREAKDOWN: return "breakdown";
    case GKO_TIMEOUT: return "timeout";
    case GKO_CUDA_ERROR: return "CUDA error";
    case GKO_BUDGET_EXCEEDED: return "memory budget exceeded";
    case GKO_NOT_SUPPORTED: return "not supported";
  }
  return "unknown status";
}

int gko_version(void) { return 100; }

int gko_device_status(void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  int* w = gko::device_error_word();
  if (!w) return gko::fail(GKO_CUDA_ERROR, "device error word unavailable");
  int v = 0;
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  GKO_TRY_CUDA(cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost));
  if (v) {
    const int zero = 0;
    GKO_TRY_CUDA(cudaMemcpy(w, &zero, sizeof(int), cudaMemcpyHostToDevice));
    if (v & (1 << GKO_TIMEOUT)) return gko::fail(GKO_TIMEOUT, "a bounded device wait timed out");
    return gko::fail(GKO_CUDA_ERROR, "device error word set");
  }
  return GKO_OK;
}

int gko_set_memory_budget(int64_t bytes) {
  if (bytes < 0) return gko::fail(GKO_INVALID_ARG, "negative budget");
  gko::g_budget.store(bytes);
  return GKO_OK;
}

int gko_memory_in_use(int64_t* in_use) {
  if (!in_use) return gko::fail(GKO_INVALID_ARG, "null in_use");
  *in_use = gko::g_in_use.load();
  return GKO_OK;
}

}  // extern "C"
