// BLAS-1 kernels and their C ABI entry points.
#include <algorithm>

#include "blas1.cuh"

namespace gko {

__device__ __forceinline__ double wide(double v) { return v; }
__device__ __forceinline__ double wide(float v) { return (double)v; }

struct StoreOp1 {
  double* result;
  __device__ void operator()(const double (&t)[1]) const { *result = t[0]; }
};

// Vector kernels are held to 64 registers (__launch_bounds__(256, 4)) and
// launched as one wave of 4 blocks per SM.  On GB300 they are FP64-pipe bound
// (about 0.5 T FMA/s for the whole GPU, measured), and at 2-4 waves of
// 64-128-register blocks the per-block prologue, barriers and reduction tail
// kept that pipe idle: 128^3 BiCGSTAB 215 -> 200 us per iteration, CG 109 ->
// 99 us, mixed BiCGSTAB 177 -> 154 us, GMRES(30) 431 -> 403 us.
int reduce_grid(int64_t n) {
  int64_t g = (n + 1023) / 1024;
  const int64_t cap = std::min<int64_t>((int64_t)sm_count() * 4, kDotSlots);
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

template <typename T>
__global__ void __launch_bounds__(256, 4) dot_kernel(int64_t n, const T* __restrict__ x, const T* __restrict__ y,
                                                  RedWs ws, double* result) {
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc[0] += wide(x[i]) * wide(y[i]);
  grid_reduce<256, 1>(acc, ws.partials, ws.counter, blockIdx.x, gridDim.x, StoreOp1{result});
}

template <typename T>
int dot_launch(int64_t n, const T* x, const T* y, double* result, RedWs ws, cudaStream_t s) {
  dot_kernel<T><<<reduce_grid(n), 256, 0, s>>>(n, x, y, ws, result);
  GKO_TRY_CUDA(cudaGetLastError());
  return GKO_OK;
}
template int dot_launch<double>(int64_t, const double*, const double*, double*, RedWs, cudaStream_t);
template int dot_launch<float>(int64_t, const float*, const float*, double*, RedWs, cudaStream_t);

__global__ void axpy_kernel(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __fma_rn(a, x[i], y[i]);
}

int axpy_launch(int64_t n, double a, const double* x, double* y, cudaStream_t s) {
  if (n == 0) return GKO_OK;
  const int64_t g = std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 4);
  axpy_kernel<<<(unsigned)g, 256, 0, s>>>(n, a, x, y);
  GKO_TRY_CUDA(cudaGetLastError());
  return GKO_OK;
}

// blockIdx.y = j: partial of V_j . w over this block's slice.
template <typename T>
__global__ void __launch_bounds__(256, 4) multi_dot_kernel(int64_t n, const T* __restrict__ V, int64_t ldv,
                                                        const T* __restrict__ w, double* __restrict__ partials) {
  const int j = blockIdx.y;
  const T* v = V + (int64_t)j * ldv;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += wide(v[i]) * wide(__ldg(w + i));
  const double sblk = block_sum<256>(acc);
  if (threadIdx.x == 0) partials[(int64_t)j * kMultiSlots + blockIdx.x] = sblk;
}

__global__ void __launch_bounds__(256, 4) multi_dot_finish_kernel(int g, const double* __restrict__ partials,
                                                               double* __restrict__ h) {
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < g; i += 256) acc += partials[(int64_t)j * kMultiSlots + i];
  const double t = block_sum<256>(acc);
  if (threadIdx.x == 0) h[j] = t;
}

template <typename T>
int multi_dot_launch(int64_t n, int32_t k, const T* V, int64_t ldv, const T* w, double* h, double* partials,
                     cudaStream_t s) {
  if (k <= 0) return GKO_OK;
  int64_t g = (n + 2047) / 2048;
  g = std::max<int64_t>(1, std::min<int64_t>(g, kMultiSlots));
  multi_dot_kernel<T><<<dim3((unsigned)g, (unsigned)k), 256, 0, s>>>(n, V, ldv, w, partials);
  multi_dot_finish_kernel<<<(unsigned)k, 256, 0, s>>>((int)g, partials, h);
  GKO_TRY_CUDA(cudaGetLastError());
  return GKO_OK;
}
template int multi_dot_launch<double>(int64_t, int32_t, const double*, int64_t, const double*, double*, double*,
                                      cudaStream_t);
template int multi_dot_launch<float>(int64_t, int32_t, const float*, int64_t, const float*, double*, double*,
                                     cudaStream_t);

template <typename T>
__global__ void __launch_bounds__(256, 4) multi_axpy_norm_kernel(int64_t n, int32_t k, const double* __restrict__ h,
                                                              const T* __restrict__ V, int64_t ldv,
                                                              T* __restrict__ y, RedWs ws, double* result) {
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = wide(y[i]);
    for (int32_t j = 0; j < k; ++j) v = __fma_rn(-__ldg(h + j), wide(V[(int64_t)j * ldv + i]), v);
    const T out = (T)v;
    y[i] = out;
    acc[0] += wide(out) * wide(out);
  }
  grid_reduce<256, 1>(acc, ws.partials, ws.counter, blockIdx.x, gridDim.x, StoreOp1{result});
}

template <typename T>
int multi_axpy_norm_launch(int64_t n, int32_t k, const double* h, const T* V, int64_t ldv, T* y, double* result,
                           RedWs ws, cudaStream_t s) {
  multi_axpy_norm_kernel<T><<<reduce_grid(n), 256, 0, s>>>(n, k, h, V, ldv, y, ws, result);
  GKO_TRY_CUDA(cudaGetLastError());
  return GKO_OK;
}
template int multi_axpy_norm_launch<double>(int64_t, int32_t, const double*, const double*, int64_t, double*,
                                            double*, RedWs, cudaStream_t);
template int multi_axpy_norm_launch<float>(int64_t, int32_t, const double*, const float*, int64_t, float*, double*,
                                           RedWs, cudaStream_t);

// Scratch layout for the entry points below: [result(s) | counter | partials].
struct AbiScratch {
  Scratch mem;
  double* result = nullptr;
  unsigned* counter = nullptr;
  double* partials = nullptr;
  int init(cudaStream_t s, int n_results, size_t partial_count) {
    const size_t head = 256 + sizeof(double) * (size_t)n_results;
    const size_t bytes = head + 256 + sizeof(double) * partial_count;
    GKO_TRY(mem.get(bytes, s));
    result = mem.as<double>(256);
    counter = mem.as<unsigned>((head + 255) / 256 * 256);
    partials = mem.as<double>((head + 255) / 256 * 256 + 256);
    GKO_TRY_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));
    return GKO_OK;
  }
  RedWs ws() const { return RedWs{partials, counter}; }
};

static int read_back(double* host, const double* dev, int count, cudaStream_t s) {
  GKO_TRY_CUDA(cudaMemcpyAsync(host, dev, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  return GKO_OK;
}

}  // namespace gko

using namespace gko;

extern "C" {

int gko_dot(int64_t n, const double* x, const double* y, double* result, void* stream) {
  if (n < 0 || !result || (n > 0 && (!x || !y))) return fail(GKO_INVALID_ARG, "bad dot arguments");
  cudaStream_t s = (cudaStream_t)stream;
  AbiScratch w;
  GKO_TRY(w.init(s, 1, kDotSlots));
  GKO_TRY(dot_launch<double>(n, x, y, w.result, w.ws(), s));
  return read_back(result, w.result, 1, s);
}

int gko_nrm2(int64_t n, const double* x, double* result, void* stream) {
  double sq = 0.0;
  GKO_TRY(gko_dot(n, x, x, &sq, stream));
  *result = sqrt(sq);
  return GKO_OK;
}

int gko_axpy(int64_t n, double a, const double* x, double* y, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return fail(GKO_INVALID_ARG, "bad axpy arguments");
  return axpy_launch(n, a, x, y, (cudaStream_t)stream);
}

int gko_multi_dot(int64_t n, int32_t k, const double* V, int64_t ldv, const double* w, double* h, void* stream) {
  if (n < 0 || k < 0 || k > 65535 || ldv < n || (k > 0 && (!V || !w || !h)))
    return fail(GKO_INVALID_ARG, "bad multi_dot arguments");
  if (k == 0) return GKO_OK;
  cudaStream_t s = (cudaStream_t)stream;
  AbiScratch sc;
  GKO_TRY(sc.init(s, k, (size_t)k * kMultiSlots));
  GKO_TRY(multi_dot_launch<double>(n, k, V, ldv, w, sc.result, sc.partials, s));
  return read_back(h, sc.result, k, s);
}

int gko_multi_axpy_norm(int64_t n, int32_t k, const double* h, const double* V, int64_t ldv, double* y,
                        double* result, void* stream) {
  if (n < 0 || k < 0 || ldv < n || !result || (n > 0 && !y) || (k > 0 && (!h || !V)))
    return fail(GKO_INVALID_ARG, "bad multi_axpy_norm arguments");
  cudaStream_t s = (cudaStream_t)stream;
  AbiScratch sc;
  GKO_TRY(sc.init(s, 1 + k, kDotSlots));
  double* dh = sc.result + 1;
  if (k > 0) GKO_TRY_CUDA(cudaMemcpyAsync(dh, h, sizeof(double) * k, cudaMemcpyHostToDevice, s));
  GKO_TRY(multi_axpy_norm_launch<double>(n, k, dh, V, ldv, y, sc.result, sc.ws(), s));
  double sq = 0.0;
  GKO_TRY(read_back(&sq, sc.result, 1, s));
  *result = sqrt(sq);
  return GKO_OK;
}

int gko_spmv_dot(gko_matrix A, const double* x, double* y, double* result, void* stream) {
  if (!A || !result || (A->n_rows > 0 && (!x || !y))) return fail(GKO_INVALID_ARG, "bad spmv_dot arguments");
  if (A->dtype != GKO_F64 || A->n_rows != A->n_cols) return fail(GKO_INVALID_ARG, "needs a square F64 matrix");
  cudaStream_t s = (cudaStream_t)stream;
  AbiScratch sc;
  GKO_TRY(sc.init(s, 2, 2 * kDotSlots));
  Scratch sp;
  const size_t sb = spmv_scratch_bytes(A);
  if (sb) GKO_TRY(sp.get(sb, s));
  if (spmv_fuses_dot(A)) {
    DotSpec d;
    d.w = x;
    d.partials = sc.partials;
    d.counter = sc.counter;
    d.result = sc.result;
    if (A->n_rows == 0) GKO_TRY_CUDA(cudaMemsetAsync(sc.result, 0, sizeof(double), s));
    else GKO_TRY(spmv_run(A, x, y, 1.0, 0.0, s, sp.data(), &d));
  } else {
    GKO_TRY(spmv_run(A, x, y, 1.0, 0.0, s, sp.data(), nullptr));
    GKO_TRY(dot_launch<double>(A->n_rows, x, y, sc.result, sc.ws(), s));
  }
  return read_back(result, sc.result, 1, s);
}

}  // extern "C"
