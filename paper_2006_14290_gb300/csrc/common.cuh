// Internal declarations shared by the translation units of the CUDA library.
// Nothing here is part of the C ABI (include/gko.h is).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <utility>

#include "gko.h"

namespace gko {

constexpr int kWarp = 32;

// ------------------------------------------------------------- errors ----

int fail(int status, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
void clear_error();

#define GKO_TRY_CUDA(call)                                   \
  do {                                                       \
    cudaError_t gko_e_ = (call);                             \
    if (gko_e_ != cudaSuccess) return ::gko::cuda_fail(gko_e_, #call); \
  } while (0)

#define GKO_TRY(expr)              \
  do {                             \
    int gko_s_ = (expr);           \
    if (gko_s_ != GKO_OK) return gko_s_; \
  } while (0)

// ------------------------------------------------------------- memory ----

// A device allocation owned by the library.  Counted against the memory
// budget; freed when the last reference goes.
struct DeviceBuffer {
  void* ptr = nullptr;
  size_t bytes = 0;
  ~DeviceBuffer();
};
using Buf = std::shared_ptr<DeviceBuffer>;

int alloc(size_t bytes, Buf* out);  // cudaMalloc with budget accounting
template <typename T>
inline T* ptr(const Buf& b) {
  return b ? static_cast<T*>(b->ptr) : nullptr;
}

// Stream-ordered scratch from the library's own memory pool.  Freed (back to
// the pool, stream-ordered) when the object goes out of scope.
class Scratch {
 public:
  Scratch() = default;
  ~Scratch();
  int get(size_t bytes, cudaStream_t s);
  void* data() const { return p_; }
  template <typename T>
  T* as(size_t byte_offset = 0) const {
    return reinterpret_cast<T*>(static_cast<char*>(p_) + byte_offset);
  }
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;

 private:
  void* p_ = nullptr;
  size_t bytes_ = 0;
  cudaStream_t s_ = nullptr;
};

int budget_reserve(size_t bytes);
void budget_release(size_t bytes);

int sm_count();
int* device_error_word();
size_t dtype_size(gko_dtype t);

// ------------------------------------------------------------- matrix ----

constexpr int kHistBins = 33;
constexpr int32_t kLongChunk = 1024;  // nonzeros per chunk of a long CSR row
constexpr int kRbThreads = 128;      // TMA row-block CSR kernel: threads per block
constexpr int kCooRbMaxCap = 4096;   // row-block COO: largest stage
constexpr unsigned kRbStages = 2;    // row-block kernels: shared-memory stages (double buffering)

// Dynamic shared memory of a row-block launch: barriers, kRbStages buffers
// of `cap` entries (column, value and, for COO, row) and the COO row-start
// table.
inline size_t rb_smem_need(int cap, size_t value_bytes, bool coo) {
  const size_t per = sizeof(int32_t) + value_bytes + (coo ? sizeof(int32_t) : 0);
  return 128 + (size_t)kRbStages * (size_t)cap * per + (coo ? 4 * (size_t)(4 * kRbThreads + 4) : 0);
}

// Load-balancing plan of the CSR SpMV, built from the row-length histogram.
struct CsrPlan {
  int32_t kind = 0;         // 0: subwarp, 1: TMA row-block, 2: merge path, 3: nonzero split
  int32_t S = 32;           // subwarp width for ordinary rows
  int32_t R = 4;            // rows per subwarp pass (row-block: rows per subwarp)
  int32_t cap = 2048;       // row-block kernel: nonzeros per shared-memory stage
  int32_t long_thr = 1024;  // rows longer than this use the nonzero split
  int32_t max_len = 0;
  int64_t hist[kHistBins] = {0};
  int64_t hist_nnz[kHistBins] = {0};
  int64_t n_long = 0, n_chunks = 0;
  Buf long_rows;       // int32[n_long]     row index of each long row
  Buf long_chunk_ptr;  // int32[n_long+1]   first chunk of each long row
  Buf chunk_row;       // int32[n_chunks]   row index of each chunk
  Buf chunk_start;     // int32[n_chunks]   first nonzero of each chunk
  Buf merge_x;         // int32[tiles+1]    merge-path row coordinate of each tile corner
  int64_t merge_tiles = 0;
  Buf seg_row;         // int32[tiles+1]    nonzero split: row of the first nonzero of each tile
  int64_t seg_tiles = 0;
  // COO handles: kind 1 runs the row-block kernel over the COO arrays, any
  // other kind the tiled segmented reduction.
  Buf coo_rb;          // int32[n_rb+1]     first COO entry of each row block of (128/S)*R rows
  int64_t coo_rb_n = 0;
};

}  // namespace gko

struct gko_matrix_s {
  gko_format fmt = GKO_CSR;
  gko_dtype dtype = GKO_F64;
  int64_t n_rows = 0, n_cols = 0, nnz = 0;
  int device = 0;
  // CSR
  gko::Buf row_ptr, col, val;
  gko::CsrPlan plan;
  // ELL (also the ELL part of HYBRID)
  int32_t K = 0;
  int64_t stride = 0;
  gko::Buf ell_col, ell_val;
  // COO (also the tail of HYBRID)
  int64_t coo_nnz = 0;
  gko::Buf coo_row, coo_col, coo_val;
  // SELL-P: slices of `slice` rows; sellp_sets int32[n_slices+1] (slice
  // offsets in columns), slots column-major within each slice
  int32_t slice = 0;
  int64_t n_slices = 0, sellp_slots = 0;
  gko::Buf sellp_sets, sellp_col, sellp_val;
  // cached low-precision copies used by mixed-precision solves
  std::mutex mu;
  std::map<int, gko_matrix> lowp;
  ~gko_matrix_s();
};

namespace gko {

// --------------------------------------------------------- device utils ----

template <typename V>
struct AccOf {
  using type = float;
};
template <>
struct AccOf<double> {
  using type = double;
};
template <typename V>
using acc_t = typename AccOf<V>::type;

__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
__device__ __forceinline__ T from_acc(double v);
template <>
__device__ __forceinline__ double from_acc<double>(double v) { return v; }
template <typename T>
__device__ __forceinline__ T from_accf(float v);
template <>
__device__ __forceinline__ float from_accf<float>(float v) { return v; }

__device__ __forceinline__ double madd(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float madd(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Streaming loads of matrix data (read once: evict-first) and cached loads
// of the gathered vector (kept resident in L2).
template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) {
  return __ldcs(p);
}
template <typename T>
__device__ __forceinline__ T ld_vec(const T* p) {
  return __ldg(p);
}

// Subwarp of `S` contiguous lanes (paper, Section 3.3): Rank = tid % S,
// LaneOffset = floor((tid % 32) / S) * S, Mask = (~0 >> (32 - S)) << LaneOffset.
template <int S>
__device__ __forceinline__ unsigned subwarp_mask() {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned offset = (lane / S) * S;
  return (0xffffffffu >> (32 - S)) << offset;
}

// Butterfly sum over a subwarp: log2(S) xor-shuffle steps (paper, Section 3.3
// reduce listing); every lane of the subwarp ends with the total.
template <int S, typename T>
__device__ __forceinline__ T subwarp_sum(T v, unsigned mask) {
#pragma unroll
  for (int m = S / 2; m > 0; m >>= 1) v += __shfl_xor_sync(mask, v, m, S);
  return v;
}

// Reduce-scatter over a subwarp of S lanes that each hold R partial sums (R
// rows).  The xor steps run S/2, ..., 1 as in subwarp_sum, so each row's sum
// is the same tree of lane partials as R separate butterflies and the result
// is bit-identical to them.  While a lane holds more than one value, a step
// halves them: the lane keeps the half that its rank bit selects and adds
// the partner's copy of that half.  Once one value is left, the steps are
// plain butterflies.  Adds per lane: R/2 + R/4 + ... down to one value, then
// one per remaining step, against R*log2(S) for separate butterflies (R = 4,
// S = 4: 3 instead of 8).  Returns the index of the first row whose complete
// sum this lane holds in v[0 .. max(1, R/S)).  The lanes whose low
// log2(S / min(R, S)) rank bits are zero hold distinct rows.
template <int S, int R, typename T>
__device__ __forceinline__ int subwarp_reduce_scatter(T (&v)[R], int rank) {
  int first = 0;
  int cnt = R;
#pragma unroll
  for (int m = S / 2; m > 0; m >>= 1) {
    if (cnt > 1) {
      const bool hi = (rank & m) != 0;
      const int h = cnt / 2;
#pragma unroll
      for (int j = 0; j < h; ++j) {
        const T keep = hi ? v[h + j] : v[j];
        const T give = hi ? v[j] : v[h + j];
        v[j] = keep + __shfl_xor_sync(0xffffffffu, give, m);
      }
      if (hi) first += h;
      cnt = h;
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], m);
    }
  }
  return first;
}

// Exact float -> double widening with integer operations (GB300 runs the
// F2F conversion instruction on its narrow FP64/conversion path).  Normal
// numbers, zeros, infinities and NaNs convert exactly; FP32 subnormals
// (|v| < 2^-126) become signed zero.
__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  const uint64_t mant = (uint64_t)(u & 0x7fffffu) << 29;
  const uint64_t expo = e == 0xffu ? 0x7ffull : (uint64_t)(e + 896u);
  const uint64_t bits = e == 0u ? sign : (sign | (expo << 52) | mant);
  return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double widen(double d) { return d; }

// y + a*x stored as T for an FP64 scalar a.  FP64 vectors: one FP64 FMA.
// FP32 vectors: a is applied as the float pair hi + lo (hi = fl32(a),
// lo = fl32(a - hi)) in two FP32 FMAs, so the scalar keeps FP64 accuracy
// while the arithmetic stays on GB300's FP32 pipe (its FP64 rate is about
// 1/64 of FP32).
template <typename T>
struct Lin;
template <>
struct Lin<double> {
  double a;
  __device__ explicit Lin(double a_) : a(a_) {}
  __device__ double operator()(double x, double y) const { return __fma_rn(a, x, y); }
  __device__ double scale(double x) const { return a * x; }
};
template <>
struct Lin<float> {
  float hi, lo;
  __device__ explicit Lin(double a) {
    hi = __double2float_rn(a);
    lo = __double2float_rn(a - (double)hi);
  }
  __device__ Lin(float h, float l) : hi(h), lo(l) {}
  __device__ float operator()(float x, float y) const { return __fmaf_rn(lo, x, __fmaf_rn(hi, x, y)); }
  __device__ float scale(float x) const { return __fmaf_rn(lo, x, hi * x); }
  // the pair's bits in one double (for broadcasting through shared memory)
  __device__ double pack() const { return __hiloint2double(__float_as_int(hi), __float_as_int(lo)); }
  __device__ static Lin unpack(double d) { return Lin(__int_as_float(__double2hiint(d)), __int_as_float(__double2loint(d))); }
};


inline unsigned ceil_div_u(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// programmatic stream serialization may be dispatched while its predecessor
// in the stream is still draining; it must not touch memory the predecessor
// writes before griddepcontrol.wait returns (the predecessor has completed
// and its writes are visible).  Every kernel that launch_k may launch this
// way starts with pdl_begin(): that wait, then launch_dependents, which lets
// its own successor be dispatched as soon as this grid's blocks leave.  For
// a kernel launched without the attribute the stream has already ordered the
// predecessor and the wait returns at once.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Whether launch_k uses programmatic serialization on this host thread (set
// by the solvers around their iteration launches, PdlScope).
bool& pdl_launches();
struct PdlScope {
  bool old;
  explicit PdlScope(bool on) : old(pdl_launches()) { pdl_launches() = on; }
  ~PdlScope() { pdl_launches() = old; }
  PdlScope(const PdlScope&) = delete;
  PdlScope& operator=(const PdlScope&) = delete;
};

// kern<<<grid, block, smem, s>>>(args...), with programmatic stream
// serialization when pdl_launches() is set.  Only kernels that begin with
// pdl_begin() may be launched through it.
template <typename... P, typename... A>
inline cudaError_t launch_k(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A&&... args) {
  if (!pdl_launches()) {
    kern<<<grid, block, smem, s>>>(std::forward<A>(args)...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

}  // namespace gko
