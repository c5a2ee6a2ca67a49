// Matrix handles: creation with on-device validation, the CSR load-balancing
// plan (row-length histogram -> subwarp width, nonzero split of long rows),
// the format conversions CSR -> ELL / COO / hybrid (Bell & Garland's
// layouts; the paper's Section 1 names the formats), value-precision copies,
// introspection and export.
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "scan.cuh"
#include "spmv.cuh"

gko_matrix_s::~gko_matrix_s() {
  for (auto& kv : lowp) delete kv.second;
}

namespace gko {

// ------------------------------------------------------------ kernels ----

__global__ void validate_kernel(int64_t n, int64_t nnz, int64_t n_cols, const int32_t* __restrict__ rp,
                                const int32_t* __restrict__ col, int* err) {
  const int64_t total = n + 1 > nnz ? n + 1 : nnz;
  int flags = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i <= n) {
      const int32_t a = rp[i];
      if (i == 0 && a != 0) flags |= 1;
      if (i == n && (int64_t)a != nnz) flags |= 2;
      if (i < n && a > rp[i + 1]) flags |= 4;
    }
    if (i < nnz) {
      const int32_t c = col[i];
      if (c < 0 || (int64_t)c >= n_cols) flags |= 8;
    }
  }
  if (flags) atomicOr(err, flags);
}

// Row-length histogram in log2 classes (bin 0: empty, bin b: [2^(b-1), 2^b)),
// nonzeros per class, and the longest row.
__global__ void row_stats_kernel(int64_t n, const int32_t* __restrict__ rp, unsigned long long* hist,
                                 unsigned long long* hist_nnz, int* max_len) {
  __shared__ unsigned int h[kHistBins];
  __shared__ unsigned long long hn[kHistBins];
  for (int b = threadIdx.x; b < kHistBins; b += blockDim.x) {
    h[b] = 0;
    hn[b] = 0;
  }
  __syncthreads();
  int lmax = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int len = rp[i + 1] - rp[i];
    const int b = len == 0 ? 0 : 32 - __clz(len);
    atomicAdd(&h[b], 1u);
    atomicAdd(&hn[b], (unsigned long long)len);
    lmax = max(lmax, len);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kHistBins; b += blockDim.x) {
    if (h[b]) atomicAdd(&hist[b], (unsigned long long)h[b]);
    if (hn[b]) atomicAdd(&hist_nnz[b], hn[b]);
  }
  if (lmax) atomicMax(max_len, lmax);
}

struct LongFlag {
  const int32_t* rp;
  int32_t thr;
  __device__ int64_t operator()(int64_t i) const { return (rp[i + 1] - rp[i]) > thr ? 1 : 0; }
};

struct LongChunkCount {
  const int32_t* rp;
  const int32_t* rows;
  __device__ int64_t operator()(int64_t j) const {
    const int32_t r = rows[j];
    return (rp[r + 1] - rp[r] + kLongChunk - 1) / kLongChunk;
  }
};

__global__ void long_rows_kernel(int64_t n, const int32_t* __restrict__ rp, int32_t thr,
                                 const int32_t* __restrict__ pos, int32_t* __restrict__ rows) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (rp[i + 1] - rp[i] > thr) rows[pos[i]] = (int32_t)i;
}

__global__ void chunks_kernel(int64_t n_long, const int32_t* __restrict__ rows, const int32_t* __restrict__ cptr,
                              const int32_t* __restrict__ rp, int32_t* __restrict__ chunk_row,
                              int32_t* __restrict__ chunk_start) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n_long; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rows[j];
    for (int32_t c = cptr[j]; c < cptr[j + 1]; ++c) {
      chunk_row[c] = r;
      chunk_start[c] = rp[r] + (c - cptr[j]) * kLongChunk;
    }
  }
}

// Row index of every nonzero: the last row whose start is <= k (binary search
// over row_ptr; empty rows are skipped naturally).
__device__ __forceinline__ int32_t row_of(const int32_t* __restrict__ rp, int64_t n, int64_t k) {
  int64_t lo = 0, hi = n;  // invariant: rp[lo] <= k < rp[hi]
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (rp[mid] <= k) lo = mid; else hi = mid;
  }
  return (int32_t)lo;
}

__global__ void coo_rows_kernel(int64_t n, int64_t nnz, const int32_t* __restrict__ rp, int32_t* __restrict__ row) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
    row[k] = row_of(rp, n, k);
}

// ELL fill: slot (k, i) at k*stride + i holds entry k of row i when
// k < min(len_i, K); padding gets col = -1 and value bits 0 (+0.0).
template <typename E>
__global__ void ell_fill_kernel(int64_t n, int32_t K, int64_t stride, const int32_t* __restrict__ rp,
                                const int32_t* __restrict__ col, const E* __restrict__ val,
                                int32_t* __restrict__ ecol, E* __restrict__ eval) {
  const int64_t slots = (int64_t)K * stride;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < slots; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = s / stride, i = s - k * stride;
    int32_t c = -1;
    E v = E(0);
    if (i < n) {
      const int32_t b = rp[i];
      if (k < rp[i + 1] - b) {
        c = col[b + k];
        v = val[b + k];
      }
    }
    ecol[s] = c;
    eval[s] = v;
  }
}

struct TailLen {
  const int32_t* rp;
  int32_t K;
  __device__ int64_t operator()(int64_t i) const {
    const int32_t len = rp[i + 1] - rp[i];
    return len > K ? len - K : 0;
  }
};

template <typename E>
__global__ void hyb_tail_kernel(int64_t n, int64_t nnz, int32_t K, const int32_t* __restrict__ rp,
                                const int32_t* __restrict__ col, const E* __restrict__ val,
                                const int32_t* __restrict__ tptr, int32_t* __restrict__ trow,
                                int32_t* __restrict__ tcol, E* __restrict__ tval) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = row_of(rp, n, k);
    const int64_t local = k - rp[r];
    if (local >= K) {
      const int64_t p = tptr[r] + (local - K);
      trow[p] = r;
      tcol[p] = col[k];
      tval[p] = val[k];
    }
  }
}

__global__ void len_hist_kernel(int64_t n, const int32_t* __restrict__ rp, unsigned long long* h) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[rp[i + 1] - rp[i]], 1ull);
}

template <typename To>
__device__ __forceinline__ To cvt_from_f64(double v);
template <>
__device__ __forceinline__ float cvt_from_f64<float>(double v) { return __double2float_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_from_f64<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

template <typename To>
__global__ void cvt_kernel(int64_t n, const double* __restrict__ a, To* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = cvt_from_f64<To>(a[i]);
}

__global__ void f32_to_bf16_kernel(int64_t n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

static unsigned grid_for(int64_t work, int threads = 256) {
  const int64_t cap = (int64_t)sm_count() * 16;
  int64_t g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  return (unsigned)(g < cap ? g : cap);
}

// ------------------------------------------------------------- plan -----

// Plan from the row-length histogram.
//  * Regular matrices (longest row <= 4x the mean row length m, e.g. stencils
//    and banded matrices) use the TMA row-block kernel.  With 128 threads per
//    block and stages of cap = 1024 entries (small stages keep many blocks
//    resident), S (lanes per row) is the smallest power of two with
//    (128/S)*m <= 0.9*cap (S = 1: one thread per row, no reduction), and R
//    (interleaved rows per subwarp) the largest power of two <= 4 with
//    (128/S)*R*m <= cap, so one row block fills about a stage.
//    No row is split.
//  * Skewed matrices use the nonzero split (kernel 3: equal tiles of
//    nonzeros, 8 per thread; on the power-law matrix 26% faster than the
//    merge path in FP64).  The merge path (kernel 2) and the subwarp kernel
//    with a nonzero split of long rows (kernel 0) stay available through
//    gko_matrix_set_plan; for kernel 0, S = the smallest power of two
//    (<= 32) not below the mean length of rows shorter than 1024, R = 2 rows
//    per pass, rows longer than 32*S split.
// Narrower values (FP32, BF16) halve or quarter the bytes a lane streams per
// entry while the x gather stays, so the row-block kernel runs best with a
// quarter of the FP64 lanes per row and two interleaved rows per subwarp
// (measured on the 27-point stencil and the banded matrix: 16% and 28% faster
// than the FP64 choice; unchanged where the FP64 choice is already one lane).
static void narrow_plan(CsrPlan& p) {
  if (p.kind != 1) return;
  const int32_t S = std::max<int32_t>(1, p.S / 4);
  if (S != p.S) {
    p.S = S;
    p.R = 2;
  }
}

static void choose_plan(CsrPlan& p, int64_t n) {
  int64_t nz_all = 0;
  for (int b = 0; b < kHistBins; ++b) nz_all += p.hist_nnz[b];
  const double mean_all = n ? (double)nz_all / (double)n : 0.0;
  if (n > 0 && p.max_len <= 4.0 * mean_all + 1.0) {
    p.kind = 1;
    p.cap = 1024;
    int32_t S = 1;
    while (S < 8 && (double)(kRbThreads / S) * mean_all > 0.9 * p.cap) S *= 2;
    int32_t R = 1;
    while (R < 4 && (double)(kRbThreads / S) * (2 * R) * mean_all <= p.cap) R *= 2;
    p.S = S;
    p.R = R;
    p.long_thr = INT32_MAX;
    return;
  }
  int64_t rows = 0, nz = 0;
  for (int b = 0; b <= 10; ++b) {
    rows += p.hist[b];
    nz += p.hist_nnz[b];
  }
  const double mean = rows ? (double)nz / (double)rows : 1.0;
  int32_t S = 1;
  while (S < 32 && (double)S < mean) S *= 2;
  p.kind = 3;
  p.S = S;
  p.R = 2;
  p.long_thr = INT32_MAX;  // the nonzero split needs no long-row split
}

// Row coordinate of every merge-path tile corner (diagonal t * tile, t =
// 0..tiles; the last corner is the end of the path).  Same search as the
// kernel's, once per matrix.
__global__ void merge_corners_kernel(int64_t n, int64_t nnz, int64_t tiles, int64_t tile_items,
                                     const int32_t* __restrict__ rp, int32_t* __restrict__ cx) {
  const int64_t total = n + nnz;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= tiles; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = t * tile_items < total ? t * tile_items : total;
    int64_t lo = d - nnz > 0 ? d - nnz : 0;
    int64_t hi = d < n ? d : n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((int64_t)rp[mid + 1] <= d - mid - 1)
        lo = mid + 1;
      else
        hi = mid;
    }
    cx[t] = (int32_t)lo;
  }
}

static int build_merge_corners(gko_matrix m, cudaStream_t s) {
  CsrPlan& p = m->plan;
  p.merge_x.reset();
  p.merge_tiles = 0;
  if (p.kind != 2) return GKO_OK;
  const int64_t tile_items = 256 * 8;  // the merge kernel's tile (256 threads x 8 items)
  const int64_t tiles = (m->n_rows + m->nnz + tile_items - 1) / tile_items;
  GKO_TRY(alloc(sizeof(int32_t) * (tiles + 1), &p.merge_x));
  merge_corners_kernel<<<grid_for(tiles + 1), 256, 0, s>>>(m->n_rows, m->nnz, tiles, tile_items,
                                                           ptr<int32_t>(m->row_ptr), ptr<int32_t>(p.merge_x));
  GKO_TRY_CUDA(cudaGetLastError());
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  p.merge_tiles = tiles;
  return GKO_OK;
}

// Nonzero-split tiles: row of nonzero t * tile for t < tiles (the last row
// whose pointer is <= it, which has nonzeros), and n - 1 for t = tiles.
__global__ void seg_rows_kernel(int64_t n, int64_t tiles, int64_t tile, const int32_t* __restrict__ rp,
                                int32_t* __restrict__ sr) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= tiles; t += (int64_t)gridDim.x * blockDim.x) {
    if (t == tiles) {
      sr[t] = (int32_t)(n - 1);
      continue;
    }
    const int64_t k = t * tile;
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo + 1) / 2;
      if ((int64_t)rp[mid] <= k)
        lo = mid;
      else
        hi = mid - 1;
    }
    sr[t] = (int32_t)lo;
  }
}

static int build_seg_rows(gko_matrix m, cudaStream_t s) {
  CsrPlan& p = m->plan;
  p.seg_row.reset();
  p.seg_tiles = 0;
  if (p.kind != 3 || m->nnz == 0) return GKO_OK;
  const int64_t tiles = (m->nnz + kCooTile - 1) / kCooTile;
  GKO_TRY(alloc(sizeof(int32_t) * (tiles + 1), &p.seg_row));
  seg_rows_kernel<<<grid_for(tiles + 1), 256, 0, s>>>(m->n_rows, tiles, kCooTile, ptr<int32_t>(m->row_ptr),
                                                      ptr<int32_t>(p.seg_row));
  GKO_TRY_CUDA(cudaGetLastError());
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  p.seg_tiles = tiles;
  return GKO_OK;
}

// First COO entry of each row block (rows [b*RB, (b+1)*RB)): lower bound of
// b*RB in the sorted row indices, b = 0..n_rb.
__global__ void coo_rb_kernel(int64_t nnz, int64_t n_rb, int64_t RB, const int32_t* __restrict__ row,
                              int32_t* __restrict__ rb) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b <= n_rb; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t target = b * RB;
    int64_t lo = 0, hi = nnz;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((int64_t)row[mid] < target)
        lo = mid + 1;
      else
        hi = mid;
    }
    rb[b] = (int32_t)lo;
  }
}

// Row-block starts of a COO handle whose plan selects the row-block kernel.
static int build_coo_rb(gko_matrix m, cudaStream_t s) {
  CsrPlan& p = m->plan;
  p.coo_rb.reset();
  p.coo_rb_n = 0;
  if (m->fmt != GKO_COO || p.kind != 1) return GKO_OK;
  const int64_t RB = (int64_t)(kRbThreads / p.S) * p.R;
  const int64_t n_rb = (m->n_rows + RB - 1) / RB;
  GKO_TRY(alloc(sizeof(int32_t) * (n_rb + 1), &p.coo_rb));
  coo_rb_kernel<<<grid_for(n_rb + 1), 256, 0, s>>>(m->coo_nnz, n_rb, RB, ptr<int32_t>(m->coo_row),
                                                    ptr<int32_t>(p.coo_rb));
  GKO_TRY_CUDA(cudaGetLastError());
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  p.coo_rb_n = n_rb;
  return GKO_OK;
}

static bool valid_S(int s) { return s == 1 || s == 2 || s == 4 || s == 8 || s == 16 || s == 32; }
static bool valid_R(int r) { return r == 1 || r == 2 || r == 4; }

static int build_long_split(gko_matrix m, cudaStream_t s) {
  CsrPlan& p = m->plan;
  p.n_long = p.n_chunks = 0;
  p.long_rows.reset();
  p.long_chunk_ptr.reset();
  p.chunk_row.reset();
  p.chunk_start.reset();
  if (p.max_len <= p.long_thr || m->n_rows == 0) return GKO_OK;
  const int32_t* rp = ptr<int32_t>(m->row_ptr);
  const int64_t n = m->n_rows;
  Buf pos;
  GKO_TRY(alloc(sizeof(int32_t) * (n + 1), &pos));
  int64_t n_long = 0;
  GKO_TRY(exclusive_scan(LongFlag{rp, p.long_thr}, n, ptr<int32_t>(pos), &n_long, s));
  GKO_TRY(alloc(sizeof(int32_t) * (n_long + 1), &p.long_rows));
  long_rows_kernel<<<grid_for(n), 256, 0, s>>>(n, rp, p.long_thr, ptr<int32_t>(pos), ptr<int32_t>(p.long_rows));
  GKO_TRY_CUDA(cudaGetLastError());
  GKO_TRY(alloc(sizeof(int32_t) * (n_long + 1), &p.long_chunk_ptr));
  int64_t n_chunks = 0;
  GKO_TRY(exclusive_scan(LongChunkCount{rp, ptr<int32_t>(p.long_rows)}, n_long, ptr<int32_t>(p.long_chunk_ptr),
                         &n_chunks, s));
  GKO_TRY(alloc(sizeof(int32_t) * (n_chunks + 1), &p.chunk_row));
  GKO_TRY(alloc(sizeof(int32_t) * (n_chunks + 1), &p.chunk_start));
  chunks_kernel<<<grid_for(n_long), 256, 0, s>>>(n_long, ptr<int32_t>(p.long_rows), ptr<int32_t>(p.long_chunk_ptr),
                                                  rp, ptr<int32_t>(p.chunk_row), ptr<int32_t>(p.chunk_start));
  GKO_TRY_CUDA(cudaGetLastError());
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  p.n_long = n_long;
  p.n_chunks = n_chunks;
  return GKO_OK;
}

static int build_plan(gko_matrix m, cudaStream_t s) {
  CsrPlan& p = m->plan;
  const int64_t n = m->n_rows;
  Scratch st;
  GKO_TRY(st.get(sizeof(unsigned long long) * 2 * kHistBins + 16, s));
  unsigned long long* dh = st.as<unsigned long long>();
  int* dmax = reinterpret_cast<int*>(dh + 2 * kHistBins);
  GKO_TRY_CUDA(cudaMemsetAsync(st.data(), 0, sizeof(unsigned long long) * 2 * kHistBins + 16, s));
  if (n > 0) {
    row_stats_kernel<<<grid_for(n), 256, 0, s>>>(n, ptr<int32_t>(m->row_ptr), dh, dh + kHistBins, dmax);
    GKO_TRY_CUDA(cudaGetLastError());
  }
  unsigned long long hh[2 * kHistBins];
  int mx = 0;
  GKO_TRY_CUDA(cudaMemcpyAsync(hh, dh, sizeof hh, cudaMemcpyDeviceToHost, s));
  GKO_TRY_CUDA(cudaMemcpyAsync(&mx, dmax, sizeof(int), cudaMemcpyDeviceToHost, s));
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  for (int b = 0; b < kHistBins; ++b) {
    p.hist[b] = (int64_t)hh[b];
    p.hist_nnz[b] = (int64_t)hh[kHistBins + b];
  }
  p.max_len = mx;
  choose_plan(p, n);
  if (m->dtype != GKO_F64) narrow_plan(p);
  GKO_TRY(build_merge_corners(m, s));
  GKO_TRY(build_seg_rows(m, s));
  return build_long_split(m, s);
}

static int check_csr_args(int64_t n_rows, int64_t n_cols, int64_t nnz, const void* rp, const void* col,
                          const void* val, gko_dtype dt) {
  if (n_rows < 0 || n_cols < 0 || nnz < 0) return fail(GKO_INVALID_ARG, "negative size");
  if (n_rows >= INT32_MAX || n_cols > INT32_MAX || nnz >= INT32_MAX)
    return fail(GKO_INVALID_ARG, "sizes must fit int32 indices");
  if (!rp) return fail(GKO_INVALID_ARG, "null row_ptr");
  if (nnz > 0 && (!col || !val)) return fail(GKO_INVALID_ARG, "null col/values");
  if (dt != GKO_F64 && dt != GKO_F32 && dt != GKO_BF16) return fail(GKO_INVALID_ARG, "bad dtype");
  return GKO_OK;
}

static int ell_fill(gko_matrix src, gko_matrix dst, int32_t K, cudaStream_t s) {
  const int64_t slots = (int64_t)K * dst->stride;
  const size_t vs = dtype_size(src->dtype);
  GKO_TRY(alloc(sizeof(int32_t) * slots, &dst->ell_col));
  GKO_TRY(alloc(vs * slots, &dst->ell_val));
  if (slots == 0) return GKO_OK;
  const int32_t* rp = ptr<int32_t>(src->row_ptr);
  const int32_t* col = ptr<int32_t>(src->col);
  const unsigned g = grid_for(slots);
  if (vs == 8)
    ell_fill_kernel<unsigned long long><<<g, 256, 0, s>>>(src->n_rows, K, dst->stride, rp, col,
        ptr<unsigned long long>(src->val), ptr<int32_t>(dst->ell_col), ptr<unsigned long long>(dst->ell_val));
  else if (vs == 4)
    ell_fill_kernel<unsigned int><<<g, 256, 0, s>>>(src->n_rows, K, dst->stride, rp, col,
        ptr<unsigned int>(src->val), ptr<int32_t>(dst->ell_col), ptr<unsigned int>(dst->ell_val));
  else
    ell_fill_kernel<unsigned short><<<g, 256, 0, s>>>(src->n_rows, K, dst->stride, rp, col,
        ptr<unsigned short>(src->val), ptr<int32_t>(dst->ell_col), ptr<unsigned short>(dst->ell_val));
  GKO_TRY_CUDA(cudaGetLastError());
  return GKO_OK;
}

// SELL-P: width of slice s = longest row among rows [s*C, (s+1)*C).
struct SliceWidth {
  const int32_t* rp;
  int64_t n;
  int32_t C;
  __device__ int64_t operator()(int64_t s) const {
    int32_t w = 0;
    const int64_t i1 = (s + 1) * C < n ? (s + 1) * C : n;
    for (int64_t i = s * C; i < i1; ++i) w = max(w, rp[i + 1] - rp[i]);
    return w;
  }
};

// SELL-P fill: thread per row slot i of the padded slice grid; entry k of
// row i at (sets[s] + k) * C + i % C, padding col = -1 and value bits 0.
template <typename E>
__global__ void sellp_fill_kernel(int64_t n, int64_t n_slices, int32_t C, const int32_t* __restrict__ rp,
                                  const int32_t* __restrict__ col, const E* __restrict__ val,
                                  const int32_t* __restrict__ sets, int32_t* __restrict__ scol,
                                  E* __restrict__ sval) {
  const int64_t rows = n_slices * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = i / C, lr = i - sl * C;
    const int64_t base = sets[sl];
    const int32_t w = sets[sl + 1] - sets[sl];
    const int32_t r0 = i < n ? rp[i] : 0;
    const int32_t len = i < n ? rp[i + 1] - r0 : 0;
    for (int32_t k = 0; k < w; ++k) {
      const int64_t q = (base + k) * C + lr;
      scol[q] = k < len ? col[r0 + k] : -1;
      sval[q] = k < len ? val[r0 + k] : E(0);
    }
  }
}

static gko_matrix new_like(gko_matrix src, gko_format fmt) {
  gko_matrix m = new gko_matrix_s();
  m->fmt = fmt;
  m->dtype = src->dtype;
  m->n_rows = src->n_rows;
  m->n_cols = src->n_cols;
  m->nnz = src->nnz;
  m->device = src->device;
  return m;
}

static int64_t round_up32(int64_t n) { return (n + 31) / 32 * 32; }

}  // namespace gko

using namespace gko;

extern "C" {

int gko_matrix_create_csr(int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t* row_ptr,
                          const int32_t* col_idx, const void* values, gko_dtype dtype,
                          int values_on_device, void* stream, gko_matrix* out) {
  if (!out) return fail(GKO_INVALID_ARG, "null out");
  *out = nullptr;
  GKO_TRY(check_csr_args(n_rows, n_cols, nnz, row_ptr, col_idx, values, dtype));
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<gko_matrix_s> m(new gko_matrix_s());
  m->fmt = GKO_CSR;
  m->dtype = dtype;
  m->n_rows = n_rows;
  m->n_cols = n_cols;
  m->nnz = nnz;
  GKO_TRY_CUDA(cudaGetDevice(&m->device));
  const size_t vs = dtype_size(dtype);
  GKO_TRY(alloc(sizeof(int32_t) * (n_rows + 1), &m->row_ptr));
  GKO_TRY(alloc(sizeof(int32_t) * nnz, &m->col));
  GKO_TRY(alloc(vs * nnz, &m->val));
  const cudaMemcpyKind kind = values_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  GKO_TRY_CUDA(cudaMemcpyAsync(m->row_ptr->ptr, row_ptr, sizeof(int32_t) * (n_rows + 1), kind, s));
  if (nnz > 0) {
    GKO_TRY_CUDA(cudaMemcpyAsync(m->col->ptr, col_idx, sizeof(int32_t) * nnz, kind, s));
    GKO_TRY_CUDA(cudaMemcpyAsync(m->val->ptr, values, vs * nnz, kind, s));
  }
  Scratch err;
  GKO_TRY(err.get(sizeof(int), s));
  GKO_TRY_CUDA(cudaMemsetAsync(err.data(), 0, sizeof(int), s));
  validate_kernel<<<grid_for(std::max<int64_t>(n_rows + 1, nnz)), 256, 0, s>>>(
      n_rows, nnz, n_cols, ptr<int32_t>(m->row_ptr), ptr<int32_t>(m->col), err.as<int>());
  GKO_TRY_CUDA(cudaGetLastError());
  int flags = 0;
  GKO_TRY_CUDA(cudaMemcpyAsync(&flags, err.data(), sizeof(int), cudaMemcpyDeviceToHost, s));
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  if (flags) {
    char msg[200];
    snprintf(msg, sizeof msg, "malformed CSR:%s%s%s%s", (flags & 1) ? " row_ptr[0]!=0" : "",
             (flags & 2) ? " row_ptr[n]!=nnz" : "", (flags & 4) ? " row_ptr decreasing" : "",
             (flags & 8) ? " column index out of range" : "");
    return fail(GKO_INVALID_ARG, msg);
  }
  GKO_TRY(build_plan(m.get(), s));
  *out = m.release();
  return GKO_OK;
}

int gko_matrix_plan(gko_matrix m, int32_t* kernel, int32_t* S, int32_t* R, int32_t* cap, int32_t* thr,
                    int64_t* n_long, int64_t* n_chunks, int64_t* hist33) {
  if (!m || (m->fmt != GKO_CSR && m->fmt != GKO_COO)) return fail(GKO_INVALID_ARG, "plan needs a CSR or COO handle");
  if (kernel) *kernel = m->plan.kind;
  if (S) *S = m->plan.S;
  if (R) *R = m->plan.R;
  if (cap) *cap = m->plan.cap;
  if (thr) *thr = m->plan.long_thr;
  if (n_long) *n_long = m->plan.n_long;
  if (n_chunks) *n_chunks = m->plan.n_chunks;
  if (hist33)
    for (int b = 0; b < kHistBins; ++b) hist33[b] = m->plan.hist[b];
  return GKO_OK;
}

int gko_matrix_set_plan(gko_matrix m, int32_t kernel, int32_t S, int32_t R, int32_t cap, void* stream) {
  if (m && m->fmt == GKO_COO) {
    const bool rb = kernel == 1;
    if (kernel < 0 || kernel > 2 || (rb && (!valid_S(S) || S > 8 || !valid_R(R) || cap < 512 || cap > kCooRbMaxCap ||
                                            (cap & (cap - 1)))))
      return fail(GKO_INVALID_ARG,
                  "COO plan: kernel 1 (row-block: S 1..8, R 1,2,4, cap 512..4096, powers of 2) or 0/2 "
                  "(segmented reduction)");
    std::lock_guard<std::mutex> lk(m->mu);
    m->plan.kind = rb ? 1 : 0;
    if (rb) {
      m->plan.S = S;
      m->plan.R = R;
      m->plan.cap = cap;
    }
    GKO_TRY(build_coo_rb(m, (cudaStream_t)stream));
    for (auto& kv : m->lowp) {  // low-precision copies share the pattern
      CsrPlan& q = kv.second->plan;
      q.kind = m->plan.kind;
      q.S = m->plan.S;
      q.R = m->plan.R;
      q.cap = m->plan.cap;
      q.coo_rb = m->plan.coo_rb;
      q.coo_rb_n = m->plan.coo_rb_n;
    }
    return GKO_OK;
  }
  if (!m || m->fmt != GKO_CSR) return fail(GKO_INVALID_ARG, "plan needs a CSR or COO handle");
  const bool rb = kernel == 1;
  if ((kernel < 0 || kernel > 3) || !valid_S(S) || !valid_R(R) || (rb && S > 8) ||
      (rb && (cap < 512 || cap > 8192 || (cap & (cap - 1)))))
    return fail(GKO_INVALID_ARG,
                "kernel 0 (subwarp: S 1..32, R 1,2,4), 1 (row-block: S 1..8, R 1,2,4, cap 512..8192, powers of 2), "
                "2 (merge path) or 3 (nonzero split)");
  std::lock_guard<std::mutex> lk(m->mu);
  m->plan.kind = kernel;
  m->plan.S = S;
  m->plan.R = R;
  if (rb) m->plan.cap = cap;
  m->plan.long_thr = kernel == 0 ? 32 * S : INT32_MAX;
  GKO_TRY(build_merge_corners(m, (cudaStream_t)stream));
  GKO_TRY(build_seg_rows(m, (cudaStream_t)stream));
  GKO_TRY(build_long_split(m, (cudaStream_t)stream));
  for (auto& kv : m->lowp) {  // low-precision copies share the pattern
    if (kv.second->fmt == GKO_CSR) {
      CsrPlan& q = kv.second->plan;
      q.kind = m->plan.kind;
      q.S = S;
      q.R = R;
      q.cap = m->plan.cap;
      q.long_thr = m->plan.long_thr;
      q.n_long = m->plan.n_long;
      q.n_chunks = m->plan.n_chunks;
      q.long_rows = m->plan.long_rows;
      q.long_chunk_ptr = m->plan.long_chunk_ptr;
      q.chunk_row = m->plan.chunk_row;
      q.chunk_start = m->plan.chunk_start;
      q.merge_x = m->plan.merge_x;
      q.merge_tiles = m->plan.merge_tiles;
      q.seg_row = m->plan.seg_row;
      q.seg_tiles = m->plan.seg_tiles;
    }
  }
  return GKO_OK;
}

int gko_matrix_convert_to_ell(gko_matrix csr, double max_fill, void* stream, gko_matrix* out) {
  if (!csr || !out) return fail(GKO_INVALID_ARG, "null argument");
  if (csr->fmt != GKO_CSR) return fail(GKO_INVALID_ARG, "conversion source must be CSR");
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t K = csr->plan.max_len;
  if (max_fill <= 0) max_fill = 8.0;
  if ((double)K * (double)csr->n_rows > max_fill * (double)std::max<int64_t>(csr->nnz, 1)) {
    char msg[160];
    snprintf(msg, sizeof msg, "ELL padding: %lld rows x width %d exceeds %.1f x nnz (%lld)",
             (long long)csr->n_rows, K, max_fill, (long long)csr->nnz);
    return fail(GKO_FORMAT_UNSUITABLE, msg);
  }
  std::unique_ptr<gko_matrix_s> m(new_like(csr, GKO_ELL));
  m->K = K;
  m->stride = round_up32(csr->n_rows);
  GKO_TRY(ell_fill(csr, m.get(), K, s));
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  *out = m.release();
  return GKO_OK;
}

int gko_matrix_convert_to_sellp(gko_matrix csr, int32_t slice_size, double max_fill, void* stream,
                                gko_matrix* out) {
  if (!csr || !out) return fail(GKO_INVALID_ARG, "null argument");
  if (csr->fmt != GKO_CSR) return fail(GKO_INVALID_ARG, "conversion source must be CSR");
  *out = nullptr;
  const int32_t C = slice_size <= 0 ? 64 : slice_size;
  if (C != 32 && C != 64 && C != 128 && C != 256) return fail(GKO_INVALID_ARG, "slice_size must be 32, 64, 128 or 256");
  if (max_fill <= 0) max_fill = 8.0;
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<gko_matrix_s> m(new_like(csr, GKO_SELLP));
  const int64_t n = csr->n_rows;
  const int64_t ns = (n + C - 1) / C;
  GKO_TRY(alloc(sizeof(int32_t) * (ns + 1), &m->sellp_sets));
  int64_t total = 0;
  GKO_TRY(exclusive_scan(SliceWidth{ptr<int32_t>(csr->row_ptr), n, C}, ns, ptr<int32_t>(m->sellp_sets), &total, s));
  if (total > INT32_MAX) return fail(GKO_FORMAT_UNSUITABLE, "SELL-P slice widths exceed int32");
  const int64_t slots = total * C;
  if ((double)slots > max_fill * (double)std::max<int64_t>(csr->nnz, 1)) {
    char msg[160];
    snprintf(msg, sizeof msg, "SELL-P padding: %lld slots exceed %.1f x nnz (%lld)", (long long)slots, max_fill,
             (long long)csr->nnz);
    return fail(GKO_FORMAT_UNSUITABLE, msg);
  }
  const int32_t total32 = (int32_t)total;
  GKO_TRY_CUDA(cudaMemcpyAsync(ptr<int32_t>(m->sellp_sets) + ns, &total32, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  const size_t vs = dtype_size(csr->dtype);
  GKO_TRY(alloc(sizeof(int32_t) * slots, &m->sellp_col));
  GKO_TRY(alloc(vs * slots, &m->sellp_val));
  if (slots > 0) {
    const int32_t* rp = ptr<int32_t>(csr->row_ptr);
    const int32_t* col = ptr<int32_t>(csr->col);
    const int32_t* sets = ptr<int32_t>(m->sellp_sets);
    const unsigned g = grid_for(ns * C);
    if (vs == 8)
      sellp_fill_kernel<unsigned long long><<<g, 256, 0, s>>>(n, ns, C, rp, col, ptr<unsigned long long>(csr->val),
          sets, ptr<int32_t>(m->sellp_col), ptr<unsigned long long>(m->sellp_val));
    else if (vs == 4)
      sellp_fill_kernel<unsigned int><<<g, 256, 0, s>>>(n, ns, C, rp, col, ptr<unsigned int>(csr->val), sets,
          ptr<int32_t>(m->sellp_col), ptr<unsigned int>(m->sellp_val));
    else
      sellp_fill_kernel<unsigned short><<<g, 256, 0, s>>>(n, ns, C, rp, col, ptr<unsigned short>(csr->val), sets,
          ptr<int32_t>(m->sellp_col), ptr<unsigned short>(m->sellp_val));
    GKO_TRY_CUDA(cudaGetLastError());
  }
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  m->slice = C;
  m->n_slices = ns;
  m->sellp_slots = slots;
  m->K = csr->plan.max_len;  // the widest slice
  m->stride = C;
  *out = m.release();
  return GKO_OK;
}

int gko_matrix_convert_to_coo(gko_matrix csr, void* stream, gko_matrix* out) {
  if (!csr || !out) return fail(GKO_INVALID_ARG, "null argument");
  if (csr->fmt != GKO_CSR) return fail(GKO_INVALID_ARG, "conversion source must be CSR");
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<gko_matrix_s> m(new_like(csr, GKO_COO));
  const int64_t nnz = csr->nnz;
  const size_t vs = dtype_size(csr->dtype);
  m->coo_nnz = nnz;
  // regular row lengths: the row-block kernel with the CSR plan's S, R, cap;
  // otherwise the tiled segmented reduction
  m->plan.max_len = csr->plan.max_len;
  for (int b = 0; b < kHistBins; ++b) {
    m->plan.hist[b] = csr->plan.hist[b];
    m->plan.hist_nnz[b] = csr->plan.hist_nnz[b];
  }
  // default: the tiled segmented reduction (measured faster than the
  // row-block schedule on COO for stencil rows); the row-block kernel is
  // chosen through gko_matrix_set_plan
  m->plan.kind = 0;
  m->plan.long_thr = INT32_MAX;
  m->plan.S = csr->plan.S;
  m->plan.R = csr->plan.R;
  m->plan.cap = std::min<int32_t>(csr->plan.cap, kCooRbMaxCap);
  GKO_TRY(alloc(sizeof(int32_t) * nnz, &m->coo_row));
  GKO_TRY(alloc(sizeof(int32_t) * nnz, &m->coo_col));
  GKO_TRY(alloc(vs * nnz, &m->coo_val));
  if (nnz > 0) {
    coo_rows_kernel<<<grid_for(nnz), 256, 0, s>>>(csr->n_rows, nnz, ptr<int32_t>(csr->row_ptr),
                                                   ptr<int32_t>(m->coo_row));
    GKO_TRY_CUDA(cudaGetLastError());
    GKO_TRY_CUDA(cudaMemcpyAsync(m->coo_col->ptr, csr->col->ptr, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, s));
    GKO_TRY_CUDA(cudaMemcpyAsync(m->coo_val->ptr, csr->val->ptr, vs * nnz, cudaMemcpyDeviceToDevice, s));
  }
  GKO_TRY(build_coo_rb(m.get(), s));
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  *out = m.release();
  return GKO_OK;
}

int gko_matrix_convert_to_hybrid(gko_matrix csr, int32_t ell_width, void* stream, gko_matrix* out) {
  if (!csr || !out) return fail(GKO_INVALID_ARG, "null argument");
  if (csr->fmt != GKO_CSR) return fail(GKO_INVALID_ARG, "conversion source must be CSR");
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = csr->n_rows;
  int32_t K = ell_width;
  if (K < 0) {
    // Bell & Garland width: largest k with #{len >= k} >= max(4096, n/3)
    const int32_t L = csr->plan.max_len;
    Scratch h;
    GKO_TRY(h.get(sizeof(unsigned long long) * (L + 1), s));
    GKO_TRY_CUDA(cudaMemsetAsync(h.data(), 0, sizeof(unsigned long long) * (L + 1), s));
    if (n > 0) {
      len_hist_kernel<<<grid_for(n), 256, 0, s>>>(n, ptr<int32_t>(csr->row_ptr), h.as<unsigned long long>());
      GKO_TRY_CUDA(cudaGetLastError());
    }
    std::vector<unsigned long long> hh(L + 1);
    GKO_TRY_CUDA(cudaMemcpyAsync(hh.data(), h.data(), sizeof(unsigned long long) * (L + 1), cudaMemcpyDeviceToHost, s));
    GKO_TRY_CUDA(cudaStreamSynchronize(s));
    K = 0;
    int64_t at_least = 0;  // #{rows with len >= k}, walking k downward
    for (int32_t k = L; k >= 0; --k) {
      at_least += (int64_t)hh[k];
      if (at_least >= 4096 && 3 * at_least >= n) {
        K = k;
        break;
      }
    }
  }
  std::unique_ptr<gko_matrix_s> m(new_like(csr, GKO_HYBRID));
  m->K = K;
  m->stride = round_up32(n);
  GKO_TRY(ell_fill(csr, m.get(), K, s));
  Buf tptr;
  GKO_TRY(alloc(sizeof(int32_t) * (n + 1), &tptr));
  int64_t tail = 0;
  GKO_TRY(exclusive_scan(TailLen{ptr<int32_t>(csr->row_ptr), K}, n, ptr<int32_t>(tptr), &tail, s));
  const size_t vs = dtype_size(csr->dtype);
  m->coo_nnz = tail;
  GKO_TRY(alloc(sizeof(int32_t) * tail, &m->coo_row));
  GKO_TRY(alloc(sizeof(int32_t) * tail, &m->coo_col));
  GKO_TRY(alloc(vs * tail, &m->coo_val));
  if (tail > 0) {
    const unsigned g = grid_for(csr->nnz);
    const int32_t* rp = ptr<int32_t>(csr->row_ptr);
    const int32_t* col = ptr<int32_t>(csr->col);
    if (vs == 8)
      hyb_tail_kernel<unsigned long long><<<g, 256, 0, s>>>(n, csr->nnz, K, rp, col, ptr<unsigned long long>(csr->val),
          ptr<int32_t>(tptr), ptr<int32_t>(m->coo_row), ptr<int32_t>(m->coo_col), ptr<unsigned long long>(m->coo_val));
    else if (vs == 4)
      hyb_tail_kernel<unsigned int><<<g, 256, 0, s>>>(n, csr->nnz, K, rp, col, ptr<unsigned int>(csr->val),
          ptr<int32_t>(tptr), ptr<int32_t>(m->coo_row), ptr<int32_t>(m->coo_col), ptr<unsigned int>(m->coo_val));
    else
      hyb_tail_kernel<unsigned short><<<g, 256, 0, s>>>(n, csr->nnz, K, rp, col, ptr<unsigned short>(csr->val),
          ptr<int32_t>(tptr), ptr<int32_t>(m->coo_row), ptr<int32_t>(m->coo_col), ptr<unsigned short>(m->coo_val));
    GKO_TRY_CUDA(cudaGetLastError());
  }
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  *out = m.release();
  return GKO_OK;
}

int gko_matrix_convert_values(gko_matrix src, gko_dtype to, void* stream, gko_matrix* out) {
  if (!src || !out) return fail(GKO_INVALID_ARG, "null argument");
  *out = nullptr;
  if (to != GKO_F32 && to != GKO_BF16 && to != GKO_F64) return fail(GKO_INVALID_ARG, "bad dtype");
  const bool ok = (src->dtype == GKO_F64) || (src->dtype == GKO_F32 && to == GKO_BF16) || src->dtype == to;
  if (!ok) return fail(GKO_NOT_SUPPORTED, "only narrowing value conversions are provided");
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<gko_matrix_s> m(new gko_matrix_s());
  m->fmt = src->fmt;
  m->dtype = to;
  m->n_rows = src->n_rows;
  m->n_cols = src->n_cols;
  m->nnz = src->nnz;
  m->device = src->device;
  m->row_ptr = src->row_ptr;
  m->col = src->col;
  m->plan.kind = src->plan.kind;
  m->plan.S = src->plan.S;
  m->plan.R = src->plan.R;
  m->plan.cap = src->plan.cap;
  m->plan.long_thr = src->plan.long_thr;
  m->plan.max_len = src->plan.max_len;
  if (src->fmt == GKO_CSR && src->dtype == GKO_F64 && to != GKO_F64) narrow_plan(m->plan);
  for (int b = 0; b < kHistBins; ++b) {
    m->plan.hist[b] = src->plan.hist[b];
    m->plan.hist_nnz[b] = src->plan.hist_nnz[b];
  }
  m->plan.n_long = src->plan.n_long;
  m->plan.n_chunks = src->plan.n_chunks;
  m->plan.long_rows = src->plan.long_rows;
  m->plan.long_chunk_ptr = src->plan.long_chunk_ptr;
  m->plan.chunk_row = src->plan.chunk_row;
  m->plan.chunk_start = src->plan.chunk_start;
  m->plan.merge_x = src->plan.merge_x;
  m->plan.merge_tiles = src->plan.merge_tiles;
  m->plan.seg_row = src->plan.seg_row;
  m->plan.seg_tiles = src->plan.seg_tiles;
  m->plan.coo_rb = src->plan.coo_rb;
  m->plan.coo_rb_n = src->plan.coo_rb_n;
  m->K = src->K;
  m->stride = src->stride;
  m->ell_col = src->ell_col;
  m->coo_nnz = src->coo_nnz;
  m->coo_row = src->coo_row;
  m->coo_col = src->coo_col;
  m->slice = src->slice;
  m->n_slices = src->n_slices;
  m->sellp_slots = src->sellp_slots;
  m->sellp_sets = src->sellp_sets;
  m->sellp_col = src->sellp_col;
  auto convert = [&](const Buf& a, int64_t count, Buf* b) -> int {
    GKO_TRY(alloc(dtype_size(to) * count, b));
    if (count == 0) return GKO_OK;
    if (src->dtype == to) {
      GKO_TRY_CUDA(cudaMemcpyAsync((*b)->ptr, a->ptr, dtype_size(to) * count, cudaMemcpyDeviceToDevice, s));
    } else if (src->dtype == GKO_F64 && to == GKO_F32) {
      cvt_kernel<float><<<grid_for(count), 256, 0, s>>>(count, ptr<double>(a), ptr<float>(*b));
    } else if (src->dtype == GKO_F64) {
      cvt_kernel<__nv_bfloat16><<<grid_for(count), 256, 0, s>>>(count, ptr<double>(a), ptr<__nv_bfloat16>(*b));
    } else {
      f32_to_bf16_kernel<<<grid_for(count), 256, 0, s>>>(count, ptr<float>(a), ptr<__nv_bfloat16>(*b));
    }
    GKO_TRY_CUDA(cudaGetLastError());
    return GKO_OK;
  };
  if (src->val) GKO_TRY(convert(src->val, src->nnz, &m->val));
  if (src->ell_val) GKO_TRY(convert(src->ell_val, (int64_t)src->K * src->stride, &m->ell_val));
  if (src->coo_val) GKO_TRY(convert(src->coo_val, src->coo_nnz, &m->coo_val));
  if (src->sellp_val) GKO_TRY(convert(src->sellp_val, src->sellp_slots, &m->sellp_val));
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  *out = m.release();
  return GKO_OK;
}

int gko_matrix_info(gko_matrix m, gko_format* format, gko_dtype* dtype, int64_t* n_rows, int64_t* n_cols,
                    int64_t* nnz, int32_t* ell_width, int64_t* ell_stride, int64_t* coo_nnz, int64_t* bytes) {
  if (!m) return fail(GKO_INVALID_ARG, "null matrix");
  if (format) *format = m->fmt;
  if (dtype) *dtype = m->dtype;
  if (n_rows) *n_rows = m->n_rows;
  if (n_cols) *n_cols = m->n_cols;
  if (nnz) *nnz = m->nnz;
  if (ell_width) *ell_width = m->K;
  if (ell_stride) *ell_stride = m->stride;
  if (coo_nnz) *coo_nnz = m->fmt == GKO_SELLP ? m->sellp_slots : m->coo_nnz;
  if (bytes) {
    int64_t b = 0;
    for (const Buf* x : {&m->row_ptr, &m->col, &m->val, &m->ell_col, &m->ell_val, &m->coo_row, &m->coo_col,
                         &m->coo_val, &m->plan.long_rows, &m->plan.long_chunk_ptr, &m->plan.chunk_row,
                         &m->plan.chunk_start, &m->plan.merge_x, &m->plan.seg_row, &m->plan.coo_rb, &m->sellp_sets,
                         &m->sellp_col, &m->sellp_val})
      if (*x) b += (int64_t)(*x)->bytes;
    *bytes = b;
  }
  return GKO_OK;
}

int gko_matrix_export(gko_matrix m, int32_t* row_ptr, int32_t* col, void* val, int32_t* ell_col, void* ell_val,
                      int32_t* coo_row, int32_t* coo_col, void* coo_val, void* stream) {
  if (!m) return fail(GKO_INVALID_ARG, "null matrix");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t vs = dtype_size(m->dtype);
  auto d2h = [&](void* dst, const Buf& b, size_t bytes) -> int {
    if (dst && b && bytes) GKO_TRY_CUDA(cudaMemcpyAsync(dst, b->ptr, bytes, cudaMemcpyDeviceToHost, s));
    return GKO_OK;
  };
  if (m->fmt == GKO_CSR) {
    GKO_TRY(d2h(row_ptr, m->row_ptr, sizeof(int32_t) * (m->n_rows + 1)));
    GKO_TRY(d2h(col, m->col, sizeof(int32_t) * m->nnz));
    GKO_TRY(d2h(val, m->val, vs * m->nnz));
  }
  if (m->fmt == GKO_ELL || m->fmt == GKO_HYBRID) {
    const int64_t slots = (int64_t)m->K * m->stride;
    GKO_TRY(d2h(ell_col, m->ell_col, sizeof(int32_t) * slots));
    GKO_TRY(d2h(ell_val, m->ell_val, vs * slots));
  }
  if (m->fmt == GKO_SELLP) {
    GKO_TRY(d2h(row_ptr, m->sellp_sets, sizeof(int32_t) * (m->n_slices + 1)));
    GKO_TRY(d2h(ell_col, m->sellp_col, sizeof(int32_t) * m->sellp_slots));
    GKO_TRY(d2h(ell_val, m->sellp_val, vs * m->sellp_slots));
  }
  if (m->fmt == GKO_COO || m->fmt == GKO_HYBRID) {
    GKO_TRY(d2h(coo_row, m->coo_row, sizeof(int32_t) * m->coo_nnz));
    GKO_TRY(d2h(coo_col, m->coo_col, sizeof(int32_t) * m->coo_nnz));
    GKO_TRY(d2h(coo_val, m->coo_val, vs * m->coo_nnz));
  }
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  return GKO_OK;
}

int gko_matrix_destroy(gko_matrix m) {
  delete m;
  return GKO_OK;
}

}  // extern "C"
