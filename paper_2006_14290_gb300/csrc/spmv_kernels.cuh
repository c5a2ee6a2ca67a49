// Kernel templates behind spmv_run_{f64,f32,bf16}.  Included by exactly one
// translation unit per value type.
//
// GB300 note: FP64 arithmetic runs at about 2 FMA per clock per SM, so an
// FP64 SpMV at HBM speed can afford roughly one fully populated FMA warp
// instruction per 32 nonzeros.  The kernels below therefore keep every lane
// of an FP64 FMA busy (thread-per-row over staged data, or one FMA per
// entry in the segmented COO pass) and avoid shuffle reductions per row
// wherever the row-length histogram allows.
#pragma once

#include <algorithm>
#include <climits>
#include <type_traits>

#include "reduce.cuh"
#include "spmv.cuh"
#include "tma.cuh"

namespace gko {

// Row result: y = alpha*s + beta*y, or y = s when alpha == 1 and beta == 0
// (no extra FP64 instruction on the common path).
template <typename XT, typename AT>
__device__ __forceinline__ AT finish_row(XT* y, int64_t i, AT s, AT alpha, AT beta, bool plain) {
  if (plain) return s;
  AT v = alpha * s;
  if (beta != AT(0)) v = madd(beta, to_acc(y[i]), v);
  return v;
}

__device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }
__device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

template <typename XT>
__device__ __forceinline__ void dot_accum(const DotSpec& d, int64_t i, XT v, double& wy, double& yy) {
  const double yv = widen(v);
  wy = __fma_rn(widen(static_cast<const XT*>(d.w)[i]), yv, wy);
  if (d.want_yy) yy = __fma_rn(yv, yv, yy);
}

// The same with w[i] loaded earlier (issued when the thread takes its rows,
// so its latency overlaps the row's gathers instead of following them).
// A caller may pass the output itself as w (w = y: the dot is ||y||^2,
// GMRES's norm of A v); an early load would read y's old contents, so the
// kernels pass the row's new value instead (dot_w).
template <typename XT>
__device__ __forceinline__ XT dot_w(const DotSpec& d, const XT* y, XT w_early, XT v) {
  return static_cast<const XT*>(d.w) == y ? v : w_early;
}
template <typename XT>
__device__ __forceinline__ void dot_accum_w(const DotSpec& d, XT w, XT v, double& wy, double& yy) {
  const double yv = widen(v);
  wy = __fma_rn(widen(w), yv, wy);
  if (d.want_yy) yy = __fma_rn(yv, yv, yy);
}

// Blocks that prefetch slices of x into L2 at the start of the gather-heavy
// kernels (COO, merge path): about the first wave of blocks.
constexpr unsigned kXPrefetchBlocks = 512;

// ------------------------------------------------------------------- CSR --

template <typename VT, typename XT>
struct CsrArgs {
  int64_t n;
  const int32_t* rp;
  const int32_t* col;
  const VT* val;
  const XT* x;
  XT* y;
  acc_t<VT> alpha, beta;
  int32_t long_thr;
  bool plain;
  // row-block COO only: the row index of every entry and the first entry of
  // every row block (rb_ptr[b] = first k with row[k] >= b*RB)
  const int32_t* row = nullptr;
  const int32_t* rb_ptr = nullptr;
  int64_t n_cols = 0;  // length of x
};

// Subwarp-per-row CSR (irregular matrices): a subwarp of S lanes owns R
// consecutive rows per pass; lane `rank` reads entries rank, rank+S, ... of
// each row, loads of all R rows are issued before the gathers, then a
// log2(S)-step butterfly sums each row.  Rows longer than long_thr are
// skipped (the nonzero split handles them).
template <int S, int R, typename VT, typename XT, bool DOT>
__global__ void __launch_bounds__(256) csr_subwarp_kernel(CsrArgs<VT, XT> a, DotSpec d, int expected,
                                                          const int* gate) {
  using AT = acc_t<VT>;
  if (gated(gate)) return;
  const unsigned mask = subwarp_mask<S>();
  const int rank = threadIdx.x & (S - 1);
  const int64_t sub = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / S;
  const int64_t nsub = ((int64_t)gridDim.x * blockDim.x) / S;
  double dwy = 0.0, dyy = 0.0;
  for (int64_t row0 = sub * R; row0 < a.n; row0 += nsub * R) {
    int32_t beg[R], end[R];
    unsigned long_bits = 0;
    int32_t lmax = 0;
    int32_t p0 = __ldg(a.rp + row0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i1 = row0 + r + 1;
      const int32_t p1 = i1 <= a.n ? __ldg(a.rp + i1) : p0;
      beg[r] = p0;
      if (p1 - p0 > a.long_thr) {
        end[r] = p0;
        long_bits |= 1u << r;
      } else {
        end[r] = p1;
        lmax = max(lmax, p1 - p0);
      }
      p0 = p1;
    }
    AT sum[R];
#pragma unroll
    for (int r = 0; r < R; ++r) sum[r] = AT(0);
    for (int off = rank; off < lmax; off += S) {
      int32_t c[R];
      VT v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int32_t k = beg[r] + off;
        const bool ok = k < end[r];
        c[r] = ok ? ld_stream(a.col + k) : -1;
        v[r] = ok ? ld_stream(a.val + k) : VT(0);
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (c[r] >= 0) sum[r] = madd(to_acc(v[r]), to_acc(ld_vec(a.x + c[r])), sum[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) sum[r] = subwarp_sum<S>(sum[r], mask);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i = row0 + r;
      if ((r & (S - 1)) == rank && i < a.n && !((long_bits >> r) & 1u)) {
        const XT v = (XT)finish_row(a.y, i, sum[r], a.alpha, a.beta, a.plain);
        a.y[i] = v;
        if (DOT) dot_accum(d, i, v, dwy, dyy);
      }
    }
  }
  if (DOT) dot_epilogue2<256>(dwy, dyy, d, blockIdx.x, expected);
}

// TMA row-block CSR (regular matrices).  A 128-thread block owns row blocks
// of RB = (128/S)*R consecutive rows (round robin over a persistent grid):
// subwarp g (S lanes) sums rows g, g + 128/S, ..., R rows interleaved.  The
// nonzeros of a row block, [row_ptr[b*RB], row_ptr[(b+1)*RB]) widened to
// 8-entry granules, stream into shared memory by bulk copies in stages of
// `cap` entries, double buffered: thread 0 issues the copy of stage q+2 while
// all threads consume stage q.  The plan sizes RB so that a typical row
// block fits one stage, so every thread has work in every stage.  Global
// loads are bulk and coalesced, and with S = 1 a row needs no reduction, so
// every FP64 FMA lane is busy.
//
// The COO variant (coo_rowblock_kernel, regular matrices in COO) keeps the
// same schedule; row blocks start at rb_ptr[b], computed once per matrix from
// the row indices.  Its stages also carry the row index of every entry, and
// before a stage is consumed the block turns those indices into the stage
// offset where each of its rows begins (sb[j] = first staged entry whose row
// is >= the block's row j, entries outside the row block clamped to the
// ends).  Row j then sums staged entries [sb[j], sb[j+1]), so no partial sum
// crosses a thread and no row needs a carry or a second launch.
template <typename VT>
inline size_t rb_smem_bytes(int cap, bool coo = false) {
  return rb_smem_need(cap, sizeof(VT), coo);
}

template <int S, int R, typename VT, typename XT, bool DOT, bool COO>
__device__ __forceinline__ void rowblock_body(const CsrArgs<VT, XT>& a, int cap, const DotSpec& d, int expected,
                                              int* err) {
  constexpr unsigned NS = kRbStages;
  using AT = acc_t<VT>;
  constexpr int G = kRbThreads / S;  // subwarps per block
  constexpr int RB = G * R;          // rows per row block
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  int32_t* scol = reinterpret_cast<int32_t*>(smem + 128);
  int32_t* srow = reinterpret_cast<int32_t*>(smem + 128 + (size_t)NS * cap * sizeof(int32_t));
  VT* sval = reinterpret_cast<VT*>(smem + 128 + (size_t)NS * cap * sizeof(int32_t) * (COO ? 2 : 1));
  int32_t* sb = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(sval) + (size_t)NS * cap * sizeof(VT));
  const int64_t nrb = (a.n + RB - 1) / RB;
  if ((int64_t)blockIdx.x >= nrb) return;
  const int tid = threadIdx.x;
  const int rank = tid & (S - 1);
  const int sg = tid / S;

  if (tid == 0) {
    for (unsigned i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
    mbar_fence_init();
  }
  __syncthreads();

  struct Cur {
    int64_t b, kb, ke, k0, k1;
    int j, nch;
  };
  auto open = [&](Cur& c) {
    const int32_t k0 = COO ? __ldg(a.rb_ptr + c.b) : __ldg(a.rp + c.b * RB);
    const int32_t k1 = COO ? __ldg(a.rb_ptr + c.b + 1) : __ldg(a.rp + min((c.b + 1) * RB, a.n));
    c.k0 = k0;
    c.k1 = k1;
    c.kb = (int64_t)(k0 & ~7);
    c.ke = ((int64_t)k1 + 7) & ~7ll;
    c.nch = (int)imax64(1, (c.ke - c.kb + cap - 1) / cap);
    c.j = 0;
  };
  auto advance = [&](Cur& c) -> bool {
    if (++c.j < c.nch) return true;
    c.b += gridDim.x;
    if (c.b >= nrb) return false;
    open(c);
    return true;
  };
  auto issue = [&](const Cur& c, int stage) {
    const int64_t cs = c.kb + (int64_t)c.j * cap;
    const int64_t len = imin64(cap, c.ke - cs);
    if (len <= 0) {
      mbar_arrive(&bar[stage]);
    } else {
      const unsigned bc = (unsigned)(len * sizeof(int32_t)), bv = (unsigned)(len * sizeof(VT));
      mbar_arrive_expect_tx(&bar[stage], (COO ? 2 * bc : bc) + bv);
      bulk_g2s(scol + (size_t)stage * cap, a.col + cs, bc, &bar[stage]);
      if (COO) bulk_g2s(srow + (size_t)stage * cap, a.row + cs, bc, &bar[stage]);
      bulk_g2s(sval + (size_t)stage * cap, a.val + cs, bv, &bar[stage]);
    }
  };

  Cur c;
  c.b = blockIdx.x;
  open(c);
  Cur p = c;
  bool p_ok = true;
  unsigned issued = 0;  // stages issued so far (thread 0)
  if (tid == 0) {
    for (unsigned i = 0; i < NS && p_ok; ++i) {
      issue(p, i);
      ++issued;
      p_ok = advance(p);
    }
  }
  int32_t rs[R], re[R];
  XT wv[R];  // fused dot: w of the subwarp's R rows, loaded with their bounds
  auto row_bounds = [&](int64_t b) {
    if (COO) return;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i = b * RB + sg + (int64_t)r * G;
      rs[r] = re[r] = 0;
      if (DOT) wv[r] = XT(0);
      if (i < a.n) {
        rs[r] = __ldg(a.rp + i);
        re[r] = __ldg(a.rp + i + 1);
        if (DOT) wv[r] = static_cast<const XT*>(d.w)[i];
      }
    }
  };
  row_bounds(c.b);
  AT sum[R];
#pragma unroll
  for (int r = 0; r < R; ++r) sum[r] = AT(0);
  double dwy = 0.0, dyy = 0.0;
  bool timed_out = false;
  for (unsigned q = 0;; ++q) {
    const int stage = (int)(q % NS);
    // Each thread waits for the stage itself; the block agrees on a time-out
    // at the barrier that ends the stage, so a stage costs one block barrier.
    const bool ok = mbar_wait(&bar[stage], (q / NS) & 1u, err);
    const int32_t* sc = scol + (size_t)stage * cap;
    const VT* sv = sval + (size_t)stage * cap;
    const int64_t cs = c.kb + (int64_t)c.j * cap;
    if (COO && ok) {
      // sb[j], j = 0..RB: first staged entry whose position is >= j, where
      // an entry's position is its row minus the block's first row, -1 for
      // entries staged before the row block and RB for entries after it (or
      // past the copied length).  Positions never decrease, so each thread
      // walks its own cap/128 consecutive entries (16-byte shared loads) and
      // writes sb only where the position changes.
      const int len = (int)imin64(cap, c.ke - cs);
      const int lo_k = (int)imax64(0, imin64(len, c.k0 - cs));
      const int hi_k = (int)imax64(0, imin64(len, c.k1 - cs));
      const int32_t base = (int32_t)(c.b * RB);
      const int32_t* sr = srow + (size_t)stage * cap;
      auto pos = [&](int k, int32_t r) -> int { return k < lo_k ? -1 : (k >= hi_k ? RB : (int)(r - base)); };
      const int E = cap / kRbThreads;  // multiple of 4 (cap >= 512)
      const int k_begin = tid * E;
      int pp = k_begin == 0 ? -1 : pos(k_begin - 1, sr[k_begin - 1]);
      for (int e = 0; e < E; e += 4) {
        const int4 v = *reinterpret_cast<const int4*>(sr + k_begin + e);
        const int k4 = k_begin + e;
        // common case: four entries of the row block, all in the row of the previous one
        if (k4 >= lo_k && k4 + 4 <= hi_k && v.w - base == pp && v.x == v.w) continue;
        const int32_t rr[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = k_begin + e + u;
          const int pk = pos(k, rr[u]);
          if (pk != pp) {
            for (int j = pp + 1; j <= pk; ++j) sb[j] = k;
            pp = pk;
          }
        }
      }
      if (tid == kRbThreads - 1)
        for (int j = pp + 1; j <= RB; ++j) sb[j] = cap;  // rows that reach the end of a full stage
    }
    if (COO) __syncthreads();  // sb complete (all threads reach it: block-uniform)
#pragma unroll
    for (int r = 0; r < R && ok; ++r) {
      const int lo = COO ? sb[sg + r * G] : (int)(imax64(rs[r], cs) - cs);
      const int hi = COO ? sb[sg + r * G + 1] : (int)(imin64(re[r], cs + cap) - cs);
      AT acc = sum[r];
      int k = lo + rank;
      for (; k + 3 * S < hi; k += 4 * S) {
        const int32_t c0 = sc[k], c1 = sc[k + S], c2 = sc[k + 2 * S], c3 = sc[k + 3 * S];
        const VT v0 = sv[k], v1 = sv[k + S], v2 = sv[k + 2 * S], v3 = sv[k + 3 * S];
        const XT x0 = ld_vec(a.x + c0), x1 = ld_vec(a.x + c1), x2 = ld_vec(a.x + c2), x3 = ld_vec(a.x + c3);
        acc = madd(to_acc(v0), to_acc(x0), acc);
        acc = madd(to_acc(v1), to_acc(x1), acc);
        acc = madd(to_acc(v2), to_acc(x2), acc);
        acc = madd(to_acc(v3), to_acc(x3), acc);
      }
      // At most 3 entries remain.  One row per subwarp: three predicated
      // steps, no loop (27-pt FP64, S = 4: 0.165 -> 0.156 ms).  With R > 1
      // the R copies of those steps cost more than the loop (banded FP64,
      // S = 4, R = 4: 0.144 -> 0.19 ms), so they keep the loop.
      if constexpr (R == 1) {
#pragma unroll
        for (int u = 0; u < 3; ++u)
          if (k + u * S < hi) acc = madd(to_acc(sv[k + u * S]), to_acc(ld_vec(a.x + sc[k + u * S])), acc);
      } else {
        for (; k < hi; k += S) acc = madd(to_acc(sv[k]), to_acc(ld_vec(a.x + sc[k])), acc);
      }
      sum[r] = acc;
    }
    // Stage consumed by everyone.  The refill below writes this buffer
    // through the async proxy (bulk copy), which the block barrier alone
    // does not order after the generic-proxy shared-memory loads above: each
    // thread first orders its own loads before later async-proxy accesses
    // (without this fence, blocks that reuse a buffer under load summed
    // entries of the next stage; seen with many row blocks per block).
    fence_proxy_async_shared();
    if (__syncthreads_or(!ok)) {
      // a wait timed out: let every copy still in flight land before the
      // block's shared memory goes
      if (tid == 0)
        for (unsigned u = q; u < issued; ++u) mbar_wait(&bar[u % NS], (u / NS) & 1u, err);
      timed_out = true;
      break;
    }
    if (tid == 0 && p_ok) {
      issue(p, stage);
      ++issued;
      p_ok = advance(p);
    }
    const bool last = c.j + 1 >= c.nch;
    if (last) {
      // Every lane of the block is here (block-uniform control flow), so the
      // full-warp mask is valid (partial-mask shuffles measured ~3x slower in
      // FP32, subwarp reduction benchmark, S = 4).  The R row sums are
      // reduce-scattered: min(R, S) lanes of the subwarp each finish
      // max(1, R/S) rows, with fewer FP64 adds than one butterfly per row.
      constexpr int W = S < R ? S : R;   // lanes holding distinct rows
      constexpr int NC = R > S ? R / S : 1;  // rows per such lane
      const int first = S > 1 ? subwarp_reduce_scatter<S, R>(sum, rank) : 0;
      if ((rank & (S / W - 1)) == 0) {
#pragma unroll
        for (int j = 0; j < NC; ++j) {
          const int64_t i = c.b * RB + sg + (int64_t)(first + j) * G;
          if (i < a.n) {
            const XT v = (XT)finish_row(a.y, i, sum[j], a.alpha, a.beta, a.plain);
            a.y[i] = v;
            if (DOT) {
              if (COO) {
                dot_accum(d, i, v, dwy, dyy);
              } else {
                XT w = wv[0];
#pragma unroll
                for (int t = 1; t < R; ++t) w = (t == first + j) ? wv[t] : w;
                dot_accum_w(d, dot_w(d, a.y, w, v), v, dwy, dyy);
              }
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) sum[r] = AT(0);
    }
    if (!advance(c)) break;
    if (last) row_bounds(c.b);
  }
  if (DOT && !timed_out) dot_epilogue2<kRbThreads>(dwy, dyy, d, blockIdx.x, expected);
}

template <int S, int R, typename VT, typename XT, bool DOT>
__global__ void __launch_bounds__(kRbThreads) csr_rowblock_kernel(CsrArgs<VT, XT> a, int cap, DotSpec d,
                                                                   int expected, const int* gate, int* err) {
  pdl_begin();
  if (gated(gate)) return;
  rowblock_body<S, R, VT, XT, DOT, false>(a, cap, d, expected, err);
}

template <int S, int R, typename VT, typename XT, bool DOT>
__global__ void __launch_bounds__(kRbThreads) coo_rowblock_kernel(CsrArgs<VT, XT> a, int cap, DotSpec d,
                                                                   int expected, const int* gate, int* err) {
  pdl_begin();
  if (gated(gate)) return;
  rowblock_body<S, R, VT, XT, DOT, true>(a, cap, d, expected, err);
}

// ------------------------------------------------- segmented tile carries --
//
// Carries of an NT-thread segmented pass (COO and merge-path kernels).  Each
// thread publishes `tail` (its sum after its last row end, or all of its sum
// without one) and whether it ended a row.  A thread that ended a row gets
// `total`, its first row's sum: `head` (its own entries of that row) plus the
// tails of the preceding threads back to the nearest one that ended a row,
// and `from_before` (no such thread: the row began before the tile).  The
// walk starts from `head` rather than from zero: 0 + t is a real FP64 add
// (signed zeros keep the compiler from folding it), and FP64 instructions
// co-limit these kernels.  The tile's last-segment sum goes to carry[2*tile+1], and also
// to carry[2*tile] when no thread ended a row.
// Every warp holding a row end (short rows): each ending thread walks back
// through shared memory, about one FP64 add per thread in total.  A warp
// without a row end (a row longer than a warp's entries) would make some
// walk long and serial, so the whole block then takes a log-step segmented
// scan instead: 5 shuffle steps per warp, then a walk over at most NT/32 - 1
// warp totals.  The choice depends only on the sparsity pattern, so results stay
// reproducible.
template <typename AT, int NT>
__device__ __forceinline__ void tile_carries(AT tail, bool has_end, AT head, AT* s_tail, int* s_end, AT* carry,
                                             int64_t tile, AT& total, bool& from_before) {
  constexpr int NW = NT / 32;
  __shared__ AT s_wv[NW];
  __shared__ int s_wf[NW];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  s_tail[t] = tail;
  s_end[t] = has_end;
  const unsigned ends = __ballot_sync(0xffffffffu, has_end);
  const bool scan = __syncthreads_or(ends == 0u);
  total = head;
  from_before = true;
  if (!scan) {
    if (has_end) {
      for (int u = t - 1; u >= 0; --u) {
        total = s_tail[u] + total;
        if (s_end[u]) {
          from_before = false;
          break;
        }
      }
    }
    if (t == 0) {
      AT tv = s_tail[NT - 1];
      bool any_end = s_end[NT - 1] != 0;
      for (int u = NT - 2; u >= 0 && !any_end; --u) {
        tv = s_tail[u] + tv;
        any_end = s_end[u] != 0;
      }
      if (!any_end) carry[2 * tile] = tv;
      carry[2 * tile + 1] = tv;
    }
    return;
  }
  // inclusive segmented scan over the warp: (f, v) combines as (f | f', f' ? v' : v + v')
  AT v = tail;
  int f = has_end;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const AT vu = __shfl_up_sync(0xffffffffu, v, d);
    const int fu = __shfl_up_sync(0xffffffffu, f, d);
    if (lane >= d) {
      if (!f) v = vu + v;
      f |= fu;
    }
  }
  if (lane == 31) {
    s_wv[w] = v;
    s_wf[w] = f;
  }
  __syncthreads();
  AT cw = AT(0);  // segment entering this warp from the warps before it
  int cf = 0;
  for (int u = w - 1; u >= 0; --u) {
    cw = s_wv[u] + cw;
    if (s_wf[u]) {
      cf = 1;
      break;
    }
  }
  AT ve = __shfl_up_sync(0xffffffffu, v, 1);  // exclusive: lanes before this one
  int fe = __shfl_up_sync(0xffffffffu, f, 1);
  if (lane == 0) {
    ve = AT(0);
    fe = 0;
  }
  if (!fe) {
    ve = cw + ve;
    fe = cf;
  }
  if (has_end) {
    total = ve + head;
    from_before = !fe;
  }
  if (t == NT - 1) {
    const AT tv = f ? v : cw + v;
    if (!(f || cf)) carry[2 * tile] = tv;
    carry[2 * tile + 1] = tv;
  }
}

// ------------------------------------------------------- merge-path CSR --
//
// Merge-path CSR (skewed matrices): the merged sequence of n row ends and
// nnz nonzeros is cut into equal pieces of kMergeItems per thread (tiles of
// 256 threads), so a row of any length spreads over as many threads and
// tiles as it needs.  The tile corners on the merge path are computed once
// per matrix (plan); a tile stages its row pointers and nonzeros in shared
// memory, each thread finds its start (row x, nonzero y) by binary search
// there, then walks its items: a nonzero adds one FMA, a row end finishes
// the row.  Rows entering a thread take the trailing partials of the
// preceding threads (tile_carries, as in the COO kernel); rows crossing tiles
// are finished by csr_merge_fixup_kernel from per-tile carries, in tile
// order.

constexpr int kMergeItems = 8;
constexpr int kMergeTile = 256 * kMergeItems;

template <typename VT, typename XT>
__global__ void __launch_bounds__(256, 5) csr_merge_kernel(CsrArgs<VT, XT> a, int64_t nnz,
                                                        const int32_t* __restrict__ corner_x,
                                                        acc_t<VT>* __restrict__ carry, const int* gate) {
  using AT = acc_t<VT>;
  __shared__ int32_t s_rp[kMergeTile + 2];  // rp[x0 .. x1 + 1] of the tile
  __shared__ int32_t s_col[kMergeTile];
  __shared__ VT s_val[kMergeTile];
  __shared__ AT s_tail[256];
  __shared__ int s_end[256];
  if (gated(gate)) return;
  prefetch_slice_l2(a.x, sizeof(XT) * (size_t)a.n_cols, kXPrefetchBlocks);
  const int t = threadIdx.x;
  const int64_t total = a.n + nnz;
  const int64_t tile = blockIdx.x;
  const int64_t dt0 = tile * kMergeTile;
  const int64_t dt1 = dt0 + kMergeTile < total ? dt0 + kMergeTile : total;
  // the tile's corners on the merge path (computed once per matrix)
  const int64_t x0 = __ldg(corner_x + tile), x1 = __ldg(corner_x + tile + 1);
  const int64_t y0 = dt0 - x0, y1 = dt1 - x1;
  const int nrows = (int)(x1 - x0), nnzt = (int)(y1 - y0);
  // stage the tile's row pointers and nonzeros (coalesced, loads first)
  for (int i = t; i <= nrows + 1; i += 256) s_rp[i] = (x0 + i <= a.n) ? __ldg(a.rp + x0 + i) : (int32_t)nnz;
#pragma unroll
  for (int h = 0; h < kMergeItems; ++h) {
    const int k = t + 256 * h;
    if (k < nnzt) {
      s_col[k] = ld_stream(a.col + y0 + k);
      s_val[k] = ld_stream(a.val + y0 + k);
    }
  }
  __syncthreads();
  const bool first_open = x0 < a.n && y0 > (int64_t)s_rp[0];
  // this thread's start inside the tile: local merge path over s_rp[1..]
  const int dl = t * kMergeItems;
  const int tile_items = (int)(dt1 - dt0);
  int xl = 0, yl = 0;
  if (dl < tile_items) {
    int lo = dl - nnzt > 0 ? dl - nnzt : 0;
    int hi = dl < nrows ? dl : nrows;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((int64_t)s_rp[mid + 1] <= y0 + (dl - mid - 1))
        lo = mid + 1;
      else
        hi = mid;
    }
    xl = lo;
    yl = dl - lo;
  }
  int items = dl < tile_items ? min(kMergeItems, tile_items - dl) : 0;
  // The thread's nonzeros are a prefix of the kMergeItems entries from yl:
  // gather their x values up front so the walk below never waits on one.
  VT pv[kMergeItems];
  XT px[kMergeItems];
#pragma unroll
  for (int u = 0; u < kMergeItems; ++u) {
    const bool in_tile = yl + u < nnzt && u < items;
    pv[u] = in_tile ? s_val[yl + u] : VT(0);
    px[u] = in_tile ? ld_vec(a.x + s_col[yl + u]) : XT(0);
  }
  AT run = AT(0), first_sum = AT(0);
  int64_t first_row = -1;
  int nends = 0;
  int64_t y = y0 + yl;
  int64_t row_end = s_rp[xl + 1];
  auto end_row = [&]() {
    const int64_t row = x0 + xl;
    if (nends == 0) {
      first_sum = run;
      first_row = row;
    } else {
      a.y[row] = (XT)finish_row(a.y, row, run, a.alpha, a.beta, a.plain);
    }
    ++nends;
    run = AT(0);
    ++xl;
    row_end = s_rp[xl + 1];
    --items;
  };
  // merge-path walk, unrolled over the thread's nonzeros (register index u)
#pragma unroll
  for (int u = 0; u < kMergeItems; ++u) {
    while (items > 0 && y >= row_end) end_row();
    if (items > 0) {
      run = madd(to_acc(pv[u]), to_acc(px[u]), run);
      ++y;
      --items;
    }
  }
  while (items > 0) end_row();
  AT tot;
  bool from_before_tile;
  tile_carries<AT, 256>(run, nends > 0, first_sum, s_tail, s_end, carry, tile, tot, from_before_tile);
  if (nends > 0) {
    if (from_before_tile && first_open)
      carry[2 * tile] = tot;
    else
      a.y[first_row] = (XT)finish_row(a.y, first_row, tot, a.alpha, a.beta, a.plain);
  }
}

// Rows that cross tiles: the tile where such a row starts adds its trailing
// partial and the first-segment partials of the following tiles.
template <typename VT, typename XT>
__global__ void __launch_bounds__(256)
    csr_merge_fixup_kernel(CsrArgs<VT, XT> a, int64_t nnz, int64_t tiles, const int32_t* __restrict__ corner_x,
                           const acc_t<VT>* __restrict__ carry, const int* gate) {
  using AT = acc_t<VT>;
  if (gated(gate)) return;
  const int64_t total = a.n + nnz;
  auto corner = [&](int64_t u, int64_t& cx, int64_t& cy) {
    const int64_t d = u * kMergeTile < total ? u * kMergeTile : total;
    cx = __ldg(corner_x + u);
    cy = d - cx;
  };
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tiles; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t xs, ys, xe, ye;
    corner(t, xs, ys);
    corner(t + 1, xe, ye);
    if (xe >= a.n) continue;
    if (!(ye > (int64_t)__ldg(a.rp + xe))) continue;  // row xe has not started: nothing open
    const bool starts_here = xe > xs || ys <= (int64_t)__ldg(a.rp + xs);
    if (!starts_here) continue;  // middle of a longer row
    AT s = carry[2 * t + 1];
    for (int64_t u = t + 1; u < tiles; ++u) {
      s += carry[2 * u];
      if (__ldg(corner_x + u + 1) > __ldg(corner_x + u)) break;  // the row ends in tile u
    }
    a.y[xe] = (XT)finish_row(a.y, xe, s, a.alpha, a.beta, a.plain);
  }
}

// Nonzero split of long rows: one warp per fixed-size chunk of a long row,
// partial sums to scratch.
template <typename VT, typename XT>
__global__ void __launch_bounds__(256)
    csr_long_chunk_kernel(int64_t n_chunks, const int32_t* __restrict__ chunk_row,
                          const int32_t* __restrict__ chunk_start, const int32_t* __restrict__ rp,
                          const int32_t* __restrict__ col, const VT* __restrict__ val, const XT* __restrict__ x,
                          acc_t<VT>* __restrict__ partial, const int* gate) {
  using AT = acc_t<VT>;
  constexpr int U = 4;
  if (gated(gate)) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < n_chunks; c += nw) {
    const int32_t r = chunk_row[c], k0 = chunk_start[c];
    const int32_t k1 = min(k0 + kLongChunk, rp[r + 1]);
    AT s = AT(0);
    for (int32_t k = k0 + lane; k < k1; k += 32 * U) {
      int32_t cc[U];
      VT vv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int32_t kk = k + 32 * u;
        const bool ok = kk < k1;
        cc[u] = ok ? ld_stream(col + kk) : -1;
        vv[u] = ok ? ld_stream(val + kk) : VT(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (cc[u] >= 0) s = madd(to_acc(vv[u]), to_acc(ld_vec(x + cc[u])), s);
    }
    s = subwarp_sum<32>(s, 0xffffffffu);
    if (lane == 0) partial[c] = s;
  }
}

// Sum each long row's chunk partials in chunk order and finish the row.
template <typename VT, typename XT, bool DOT>
__global__ void __launch_bounds__(256)
    csr_long_fixup_kernel(int64_t n_long, const int32_t* __restrict__ rows, const int32_t* __restrict__ cptr,
                          const acc_t<VT>* __restrict__ partial, XT* __restrict__ y, acc_t<VT> alpha,
                          acc_t<VT> beta, bool plain, DotSpec d, int slot, int expected, const int* gate) {
  using AT = acc_t<VT>;
  if (gated(gate)) return;
  double dwy = 0.0, dyy = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n_long; j += (int64_t)gridDim.x * blockDim.x) {
    AT s = AT(0);
    for (int32_t c = cptr[j]; c < cptr[j + 1]; ++c) s += partial[c];
    const int32_t i = rows[j];
    const XT v = (XT)finish_row(y, i, s, alpha, beta, plain);
    y[i] = v;
    if (DOT) dot_accum(d, i, v, dwy, dyy);
  }
  if (DOT) dot_epilogue2<256>(dwy, dyy, d, slot + blockIdx.x, expected);
}

// ------------------------------------------------------------------- ELL --

template <typename VT, int RPT>
struct EllVec;
template <>
struct EllVec<double, 2> {
  static __device__ __forceinline__ void load(const double* p, double (&v)[2]) {
    const double2 t = __ldcs(reinterpret_cast<const double2*>(p));
    v[0] = t.x;
    v[1] = t.y;
  }
};
template <>
struct EllVec<float, 4> {
  static __device__ __forceinline__ void load(const float* p, float (&v)[4]) {
    const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  }
};
template <>
struct EllVec<__nv_bfloat16, 4> {
  static __device__ __forceinline__ void load(const __nv_bfloat16* p, __nv_bfloat16 (&v)[4]) {
    const uint2 t = __ldcs(reinterpret_cast<const uint2*>(p));
    v[0] = __ushort_as_bfloat16((unsigned short)(t.x & 0xffffu));
    v[1] = __ushort_as_bfloat16((unsigned short)(t.x >> 16));
    v[2] = __ushort_as_bfloat16((unsigned short)(t.y & 0xffffu));
    v[3] = __ushort_as_bfloat16((unsigned short)(t.y >> 16));
  }
};

template <int RPT>
__device__ __forceinline__ void ell_cols(const int32_t* p, int32_t (&c)[RPT]);
template <>
__device__ __forceinline__ void ell_cols<2>(const int32_t* p, int32_t (&c)[2]) {
  const int2 t = __ldcs(reinterpret_cast<const int2*>(p));
  c[0] = t.x;
  c[1] = t.y;
}
template <>
__device__ __forceinline__ void ell_cols<4>(const int32_t* p, int32_t (&c)[4]) {
  const int4 t = __ldcs(reinterpret_cast<const int4*>(p));
  c[0] = t.x;
  c[1] = t.y;
  c[2] = t.z;
  c[3] = t.w;
}

template <typename VT, typename XT>
struct EllArgs {
  int64_t n;
  int32_t K;
  int64_t stride;
  const int32_t* col;
  const VT* val;
  const XT* x;
  XT* y;
  acc_t<VT> alpha, beta;
  bool plain;
  // SELL-P: slice height C = 2^cshift and slice offsets (sets[s]: first
  // column of slice s)
  int32_t C = 0, cshift = 0;
  const int32_t* sets = nullptr;
};

// Column-major ELL: each thread owns RPT consecutive rows and reads slot k of
// all of them with one 128-bit (or 64-bit) load per array; padding slots
// (col = -1) never touch x, and a thread stops at the first 4-slot chunk that
// ends in padding for all its rows.
// SELL (SELL-P): the same walk inside the thread's slice, whose own width and
// first column come from sets[]; slot k of row i is at (sets[s] + k) * C +
// i % C.  Slices of 64 rows are one warp's rows in FP64 (2 per thread), so a
// warp's trip count is its slice width.
template <int RPT, typename VT, typename XT, bool DOT, bool SELL>
__global__ void __launch_bounds__(256) ell_kernel(EllArgs<VT, XT> a, DotSpec d, int expected, const int* gate) {
  using AT = acc_t<VT>;
  constexpr int U = 4;
  pdl_begin();
  if (gated(gate)) return;
  const int64_t groups = (a.n + RPT - 1) / RPT;
  double dwy = 0.0, dyy = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = g * RPT;
    int32_t width = a.K;
    int64_t first = i0, step = a.stride;
    if (SELL) {
      const int64_t sl = i0 >> a.cshift;
      const int32_t b = __ldg(a.sets + sl);
      width = __ldg(a.sets + sl + 1) - b;
      first = ((int64_t)b << a.cshift) + (i0 & (a.C - 1));
      step = a.C;
    }
    AT sum[RPT];
    XT wv[RPT];  // fused dot: w of the thread's rows, loaded before the row sums
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      sum[r] = AT(0);
      if (DOT) wv[r] = i0 + r < a.n ? static_cast<const XT*>(d.w)[i0 + r] : XT(0);
    }
    for (int32_t k = 0; k < width; k += U) {
      int32_t c[U][RPT];
      VT v[U][RPT];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (k + u < width) {
          const int64_t off = (int64_t)(k + u) * step + first;
          ell_cols<RPT>(a.col + off, c[u]);
          EllVec<VT, RPT>::load(a.val + off, v[u]);
        } else {
#pragma unroll
          for (int r = 0; r < RPT; ++r) c[u][r] = -1;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int r = 0; r < RPT; ++r)
          if (c[u][r] >= 0) sum[r] = madd(to_acc(v[u][r]), to_acc(ld_vec(a.x + c[u][r])), sum[r]);
      // Padding is trailing in every row: once the chunk's last slot is
      // padding in all of this thread's rows, so is the rest, and the thread
      // stops loading (its lanes' sectors drop out of the warp's loads).
      bool done = true;
#pragma unroll
      for (int r = 0; r < RPT; ++r) done = done && c[U - 1][r] < 0;
      if (done) break;
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int64_t i = i0 + r;
      if (i < a.n) {
        const XT v = (XT)finish_row(a.y, i, sum[r], a.alpha, a.beta, a.plain);
        a.y[i] = v;
        if (DOT) dot_accum_w(d, dot_w(d, a.y, wv[r], v), v, dwy, dyy);
      }
    }
  }
  if (DOT) dot_epilogue2<256>(dwy, dyy, d, blockIdx.x, expected);
}

// ------------------------------------------------------------------- COO --

template <typename VT, typename XT>
struct CooArgs {
  int64_t n_rows, n_cols, nnz;
  const int32_t* row;
  const int32_t* col;
  const VT* val;
  const XT* x;
  XT* y;
  acc_t<VT> alpha, beta;
  bool plain;  // alpha == 1 and beta == 0
};

template <typename VT>
struct Load8;
template <>
struct Load8<double> {
  static __device__ __forceinline__ void run(const double* p, double* v) {
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const double2 t = __ldcs(reinterpret_cast<const double2*>(p) + h);
      v[2 * h] = t.x;
      v[2 * h + 1] = t.y;
    }
  }
};
template <>
struct Load8<float> {
  static __device__ __forceinline__ void run(const float* p, float* v) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float4 t = __ldcs(reinterpret_cast<const float4*>(p) + h);
      v[4 * h] = t.x;
      v[4 * h + 1] = t.y;
      v[4 * h + 2] = t.z;
      v[4 * h + 3] = t.w;
    }
  }
};
template <>
struct Load8<__nv_bfloat16> {
  static __device__ __forceinline__ void run(const __nv_bfloat16* p, __nv_bfloat16* v) {
    const uint4 t = __ldcs(reinterpret_cast<const uint4*>(p));
    const unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      v[2 * h] = __ushort_as_bfloat16((unsigned short)(w[h] & 0xffffu));
      v[2 * h + 1] = __ushort_as_bfloat16((unsigned short)(w[h] >> 16));
    }
  }
};
__device__ __forceinline__ void load8_i32(const int32_t* p, int32_t* v) {
  const int4 a = __ldcs(reinterpret_cast<const int4*>(p));
  const int4 b = __ldcs(reinterpret_cast<const int4*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// Combine of the segmented-sum scan: `prev` precedes `cur`; a segment end in
// `cur` cuts off everything before it.
template <typename AT>
__device__ __forceinline__ void seg_combine(int fp, AT vp, int& f, AT& v) {
  if (!f) v = vp + v;
  f = f | fp;
}

// plain: alpha == 1 and beta == 0, decided once on the host (no FP64
// compare per row on the device)
template <typename XT, typename AT>
__device__ __forceinline__ void coo_store(XT* y, int32_t r, AT s, AT alpha, AT beta, bool accum, bool plain) {
  if (accum) {
    y[r] = (XT)(alpha == AT(1) ? s + to_acc(y[r]) : madd(alpha, s, to_acc(y[r])));
  } else if (plain) {
    y[r] = (XT)s;
  } else {
    AT v = alpha * s;
    if (beta != AT(0)) v = madd(beta, to_acc(y[r]), v);
    y[r] = (XT)v;
  }
}

template <typename XT, typename AT>
__device__ __forceinline__ void coo_empty_rows(XT* y, int64_t r0, int64_t r1, AT beta) {
  for (int64_t r = r0; r < r1; ++r) y[r] = beta == AT(0) ? XT(0) : (XT)(beta * to_acc(y[r]));
}

// Resident 128-thread blocks per SM the COO kernel's register budget is held
// to: 9 for FP64 values (56 registers, the most blocks without spills), 11
// for FP32/BF16 (40 registers; at 48 without spills it ran 6-8% slower).
// FP64 against 256-thread blocks at 5 per SM (48 registers, with spills):
// 5-8% faster, a tile's block barriers waiting on 4 warps instead of 8.
template <typename VT>
constexpr int coo_min_blocks() {
  return std::is_same<VT, double>::value ? 9 : 11;
}

// One thread's pass over its entries: an FMA per entry; rows that start and
// end here are stored now.  FULL: all IPT entries are present (every thread
// of every tile but the last), so the entry guards and the next-row choice
// are compile-time.  The row-end bookkeeping is written as selects around a
// predicated store (measured the same as the branchy form).
template <bool FULL, bool ACCUM, bool PLAIN, int IPT, typename VT, typename XT, typename AT>
__device__ __forceinline__ void coo_thread_pass(const CooArgs<VT, XT>& a, const int32_t (&rows)[IPT],
                                                const int32_t (&cols)[IPT], const VT (&vals)[IPT], int my,
                                                int32_t next_row, AT& run, AT& first_sum, int32_t& first_row,
                                                int& nends) {
#pragma unroll
  for (int u = 0; u < IPT; ++u) {
    if (FULL || u < my) {
      const int32_t r = rows[u];
      run = madd(to_acc(vals[u]), to_acc(ld_vec(a.x + cols[u])), run);
      const int32_t nr = FULL ? (u + 1 < IPT ? rows[u + 1] : next_row) : (u + 1 < my ? rows[u + 1] : next_row);
      const bool e = r != nr;
      if (e && nends > 0) coo_store(a.y, r, run, a.alpha, a.beta, ACCUM, PLAIN);
      const bool f = e && nends == 0;
      first_sum = f ? run : first_sum;
      first_row = f ? r : first_row;
      nends += e ? 1 : 0;
      run = e ? AT(0) : run;
    }
  }
}

// Tiled segmented reduction over row-sorted COO.  Each block of kCooThreads
// threads owns a tile of kCooTile entries; each thread owns kCooItems consecutive
// entries (vector loads) and folds them with one FMA per entry, finishing
// the rows that start and end inside its entries on the spot.  The running
// sum entering a thread's first row is the sum of the trailing partials of
// the preceding threads back to the nearest one that ended a row
// (tile_carries).  The tile's open first/last segment partials go to
// carry[2*tile] / carry[2*tile+1] for coo_fixup_kernel.
// ACCUM: y[r] += alpha*sum (hybrid tail); otherwise rows absent from the COO
// arrays are scaled by beta here too.
// PLAIN: alpha == 1 and beta == 0, the store is a plain write (coo_launch
// picks the instantiation from a.plain).
template <typename VT, typename XT, bool ACCUM, int IPT = kCooItems, int MINB = 1, bool PLAIN = false>
__global__ void __launch_bounds__(kCooThreads, MINB) coo_kernel(CooArgs<VT, XT> a, acc_t<VT>* __restrict__ carry,
                                                                const int* gate) {
  using AT = acc_t<VT>;
  constexpr int kTile = kCooThreads * IPT;
  __shared__ AT s_tail[kCooThreads];
  __shared__ int s_end[kCooThreads];
  if (gated(gate)) return;
  prefetch_slice_l2(a.x, sizeof(XT) * (size_t)a.n_cols, kXPrefetchBlocks);
  const int t = threadIdx.x;
  const int64_t tile = blockIdx.x;
  const int64_t base = tile * kTile;
  const int cnt = (int)min((int64_t)kTile, a.nnz - base);
  const int j0 = t * IPT;
  const int my = max(0, min(IPT, cnt - j0));

  int32_t rows[IPT];
  int32_t cols[IPT];
  VT vals[IPT];
  if (my == IPT) {
#pragma unroll
    for (int h = 0; h < IPT; h += 8) {
      load8_i32(a.row + base + j0 + h, rows + h);
      load8_i32(a.col + base + j0 + h, cols + h);
      Load8<VT>::run(a.val + base + j0 + h, vals + h);
    }
  } else {
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
      if (u < my) {
        const int64_t k = base + j0 + u;
        rows[u] = a.row[k];
        cols[u] = a.col[k];
        vals[u] = a.val[k];
      } else {
        rows[u] = INT_MAX;
        cols[u] = 0;
        vals[u] = VT(0);
      }
    }
  }
  // Row of the entry after this thread's last one (-1 after the matrix's
  // last entry): the next lane's first row by a shuffle; lane 31 and the
  // tile's last thread load it.  No block barrier here (exchanging it
  // through shared memory cost 4-5% on FP64).
  const int32_t nb = __shfl_down_sync(0xffffffffu, my > 0 ? rows[0] : INT_MAX, 1);
  int32_t next_row;
  if (j0 + IPT < cnt)
    next_row = (t & 31) != 31 ? nb : a.row[base + j0 + IPT];
  else
    next_row = (base + cnt < a.nnz) ? a.row[base + cnt] : -1;
  // rows before the first entry of the matrix have no entries
  if (!ACCUM && base == 0 && t == 0 && my > 0) coo_empty_rows(a.y, 0, (int64_t)rows[0], a.beta);

  AT run = AT(0), first_sum = AT(0);
  int32_t first_row = -1;
  int nends = 0;
  if (my == IPT)
    coo_thread_pass<true, ACCUM, PLAIN>(a, rows, cols, vals, my, next_row, run, first_sum, first_row, nends);
  else
    coo_thread_pass<false, ACCUM, PLAIN>(a, rows, cols, vals, my, next_row, run, first_sum, first_row, nends);
  // Rows without entries lie between a row's end and the next entry's row;
  // the thread that owns that row end scales them by beta.  Rows are sorted,
  // so rows[0] .. stop-1 (stop: the next entry's row, or n) are all present
  // exactly when there are as many of them as row ends here; otherwise
  // (rare) the gaps are found from the row indices in memory.
  const int32_t n_rows32 = (int32_t)a.n_rows;
  const bool gap = !ACCUM && my > 0 && (next_row < 0 ? n_rows32 : next_row) - rows[0] > nends;
  if (!ACCUM && gap) {
#pragma unroll 1
    for (int u = 0; u < my; ++u) {
      const int64_t k = base + j0 + u;
      const int32_t r = a.row[k];
      const int32_t nr = (u + 1 < my) ? a.row[k + 1] : next_row;
      const int32_t gap_end = nr < 0 ? n_rows32 : nr;
      if (r != nr && r + 1 < gap_end) coo_empty_rows(a.y, (int64_t)r + 1, (int64_t)gap_end, a.beta);
    }
  }
  AT total;
  bool from_before_tile;
  tile_carries<AT, kCooThreads>(run, nends > 0, first_sum, s_tail, s_end, carry, tile, total, from_before_tile);
  if (nends > 0) {
    // the tile's first row began in an earlier tile: its sum so far is a carry
    const bool first_open = from_before_tile && base > 0 && a.row[base - 1] == a.row[base];
    if (first_open)
      carry[2 * tile] = total;
    else
      coo_store(a.y, first_row, total, a.alpha, a.beta, ACCUM, PLAIN);
  }
}

// Segmented-reduction COO pass (kernel + fix-up) on stream s, with the
// instantiation for a.plain (the hybrid tail always accumulates).
template <typename VT, typename XT, bool ACCUM>
inline void coo_launch(const CooArgs<VT, XT>& a, acc_t<VT>* carry, const int* gate, cudaStream_t s);

// Complete rows that span tiles: the tile where such a row starts adds its
// last-segment partial and the first-segment partials of the following
// tiles, in tile order.
template <typename VT, typename XT, bool ACCUM>
__global__ void __launch_bounds__(256)
    coo_fixup_kernel(int64_t nnz, int64_t tiles, const int32_t* __restrict__ row, const acc_t<VT>* __restrict__ carry,
                     XT* __restrict__ y, acc_t<VT> alpha, acc_t<VT> beta, const int* gate,
                     int64_t tile_size = kCooTile) {
  using AT = acc_t<VT>;
  if (gated(gate)) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tiles; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t * tile_size;
    const int64_t e = min(b + tile_size, nnz);  // one past the tile
    if (e >= nnz || row[e - 1] != row[e]) continue;  // last segment closed
    const bool first_open = b > 0 && row[b - 1] == row[b];
    if (first_open && row[b] == row[e - 1]) continue;  // middle of a longer row
    const int32_t r = row[e - 1];
    AT s = carry[2 * t + 1];
    for (int64_t u = t + 1; u < tiles; ++u) {
      const int64_t bu = u * tile_size, eu = min(bu + tile_size, nnz);
      s += carry[2 * u];
      const bool open = eu < nnz && row[eu - 1] == row[eu];
      if (!(open && row[bu] == row[eu - 1])) break;
    }
    coo_store(y, r, s, alpha, beta, ACCUM, alpha == acc_t<VT>(1) && beta == acc_t<VT>(0));
  }
}

template <typename VT, typename XT, bool ACCUM>
inline void coo_launch(const CooArgs<VT, XT>& a, acc_t<VT>* carry, const int* gate, cudaStream_t s) {
  constexpr int kMinB = coo_min_blocks<VT>();
  const int64_t tiles = (a.nnz + kCooTile - 1) / kCooTile;
  const unsigned fg = (unsigned)std::min<int64_t>((tiles + 255) / 256, 4096);
  if constexpr (!ACCUM) {
    if (a.plain) {
      coo_kernel<VT, XT, false, kCooItems, kMinB, true><<<(unsigned)tiles, kCooThreads, 0, s>>>(a, carry, gate);
    } else {
      coo_kernel<VT, XT, false, kCooItems, kMinB, false><<<(unsigned)tiles, kCooThreads, 0, s>>>(a, carry, gate);
    }
  } else {
    coo_kernel<VT, XT, true, kCooItems, kMinB, false><<<(unsigned)tiles, kCooThreads, 0, s>>>(a, carry, gate);
  }
  coo_fixup_kernel<VT, XT, ACCUM><<<fg, 256, 0, s>>>(a.nnz, tiles, a.row, carry, a.y, a.alpha, a.beta, gate);
}

// ------------------------------------------------- nonzero-split CSR --
//
// Nonzero-split CSR (skewed matrices): the nonzeros are cut into tiles of
// kCooTile, kCooItems consecutive ones per thread loaded with 16-byte loads,
// as in the COO kernel, but no row index is read: a row ends where the next
// row pointer lies.  The plan holds seg_row[t], the row of nonzero
// t*kCooTile (t < tiles), and seg_row[tiles] = n - 1.  A tile stages
// row_ptr[seg_row[t] .. seg_row[t+1] + 1] in shared memory (reads it from
// global memory instead when that slice is longer than kSegRpCap, i.e. the
// tile spans thousands of empty rows); each thread finds the row of its first
// nonzero by binary search there and walks its entries.  Carries as in the
// COO kernel; rows that cross tiles are finished by csr_seg_fixup_kernel.
// Rows without nonzeros are written by the thread that ends the row before
// them (those before the first nonzero by tile 0's first thread).
constexpr int kSegRpCap = 2048;

template <bool FULL, bool PLAIN, typename VT, typename XT, typename AT, typename RPV>
__device__ __forceinline__ void csr_seg_pass(const CsrArgs<VT, XT>& a, const int32_t (&cols)[kCooItems],
                                             const VT (&vals)[kCooItems], int my, int32_t k0, const RPV& rpv,
                                             int32_t r, AT& run, AT& first_sum, int32_t& first_row, int& nends) {
  const int32_t n32 = (int32_t)a.n;
  int32_t nb = rpv(r + 1);  // one past the last nonzero of row r
#pragma unroll
  for (int u = 0; u < kCooItems; ++u) {
    if (FULL || u < my) {
      run = madd(to_acc(vals[u]), to_acc(ld_vec(a.x + cols[u])), run);
      const int32_t k1 = k0 + u + 1;
      if (k1 == nb) {  // row r ends at this entry
        if (nends == 0) {
          first_sum = run;
          first_row = r;
        } else {
          coo_store(a.y, r, run, a.alpha, a.beta, false, PLAIN);
        }
        ++nends;
        run = AT(0);
        // on to the next row with nonzeros; the rows skipped have none
        ++r;
        nb = r < n32 ? rpv(r + 1) : INT_MAX;
        while (nb == k1) {
          coo_empty_rows(a.y, (int64_t)r, (int64_t)r + 1, a.beta);
          ++r;
          nb = r < n32 ? rpv(r + 1) : INT_MAX;
        }
      }
    }
  }
}

template <typename VT, typename XT, bool PLAIN>
__global__ void __launch_bounds__(kCooThreads, coo_min_blocks<VT>())
    csr_seg_kernel(CsrArgs<VT, XT> a, int64_t nnz, const int32_t* __restrict__ seg_row,
                   acc_t<VT>* __restrict__ carry, const int* gate) {
  using AT = acc_t<VT>;
  __shared__ int32_t s_rp[kSegRpCap + 2];
  __shared__ AT s_tail[kCooThreads];
  __shared__ int s_end[kCooThreads];
  if (gated(gate)) return;
  prefetch_slice_l2(a.x, sizeof(XT) * (size_t)a.n_cols, kXPrefetchBlocks);
  const int t = threadIdx.x;
  const int64_t tile = blockIdx.x;
  const int64_t base = tile * kCooTile;
  const int cnt = (int)min((int64_t)kCooTile, nnz - base);
  const int j0 = t * kCooItems;
  const int my = max(0, min(kCooItems, cnt - j0));
  int32_t cols[kCooItems];
  VT vals[kCooItems];
  if (my == kCooItems) {
    load8_i32(a.col + base + j0, cols);
    Load8<VT>::run(a.val + base + j0, vals);
  } else {
#pragma unroll
    for (int u = 0; u < kCooItems; ++u) {
      cols[u] = u < my ? a.col[base + j0 + u] : 0;
      vals[u] = u < my ? a.val[base + j0 + u] : VT(0);
    }
  }
  const int32_t ra = __ldg(seg_row + tile), rb = __ldg(seg_row + tile + 1);
  const int span = rb - ra + 2;  // row pointers ra .. rb + 1
  const bool staged = span <= kSegRpCap + 2;
  if (staged)
    for (int i = t; i < span; i += kCooThreads) s_rp[i] = __ldg(a.rp + ra + i);
  __syncthreads();
  const auto rpv = [&](int32_t r) -> int32_t { return staged ? s_rp[r - ra] : __ldg(a.rp + r); };
  // rows before the first nonzero of the matrix have none
  if (base == 0 && t == 0) coo_empty_rows(a.y, 0, (int64_t)ra, a.beta);

  const int32_t k0 = (int32_t)(base + j0);
  AT run = AT(0), first_sum = AT(0);
  int32_t first_row = -1;
  int nends = 0;
  if (my > 0) {
    int32_t lo = ra, hi = rb;  // the last row starting at or before k0 holds it
    while (lo < hi) {
      const int32_t mid = lo + (hi - lo + 1) / 2;
      if (rpv(mid) <= k0)
        lo = mid;
      else
        hi = mid - 1;
    }
    if (my == kCooItems)
      csr_seg_pass<true, PLAIN>(a, cols, vals, my, k0, rpv, lo, run, first_sum, first_row, nends);
    else
      csr_seg_pass<false, PLAIN>(a, cols, vals, my, k0, rpv, lo, run, first_sum, first_row, nends);
  }
  AT total;
  bool from_before_tile;
  tile_carries<AT, kCooThreads>(run, nends > 0, first_sum, s_tail, s_end, carry, tile, total, from_before_tile);
  if (nends > 0) {
    // the tile's first row began in an earlier tile: its sum so far is a carry
    const bool first_open = from_before_tile && rpv(first_row) < base;
    if (first_open)
      carry[2 * tile] = total;
    else
      coo_store(a.y, first_row, total, a.alpha, a.beta, false, PLAIN);
  }
}

// Rows that cross tiles: the tile where such a row begins adds its last
// segment and the first segments of the following tiles, in tile order.
template <typename VT, typename XT>
__global__ void __launch_bounds__(256)
    csr_seg_fixup_kernel(CsrArgs<VT, XT> a, int64_t tiles, const int32_t* __restrict__ seg_row,
                         const acc_t<VT>* __restrict__ carry, const int* gate) {
  using AT = acc_t<VT>;
  if (gated(gate)) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t + 1 < tiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = seg_row[t + 1];  // row of the next tile's first nonzero
    const int64_t rs = a.rp[r];
    if (rs >= (t + 1) * kCooTile) continue;  // it starts there: nothing crosses
    if (rs < t * kCooTile) continue;         // it began before this tile
    AT s = carry[2 * t + 1];
    for (int64_t u = t + 1; u < tiles; ++u) {
      s += carry[2 * u];
      if (!(u + 1 < tiles && seg_row[u + 1] == r)) break;  // row r ends in tile u
    }
    a.y[r] = (XT)finish_row(a.y, r, s, a.alpha, a.beta, a.plain);
  }
}

template <typename XT, typename AT>
__global__ void scale_kernel(int64_t n, XT* __restrict__ y, AT beta, const int* gate) {
  if (gated(gate)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = beta == AT(0) ? XT(0) : (XT)(beta * to_acc(y[i]));
}

// -------------------------------------------------------------- dispatch --

template <typename K>
int resident_blocks(K kernel, int threads, size_t smem = 0) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess || nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  return nb;
}

constexpr int kLaunchCudaError = -2;  // a launch helper's "CUDA refused", status already recorded

template <typename VT, typename XT>
struct SpmvImpl {
  using AT = acc_t<VT>;

  static CsrArgs<VT, XT> csr_args(const gko_matrix_s* A, const XT* x, XT* y, AT alpha, AT beta) {
    CsrArgs<VT, XT> a{A->n_rows, ptr<int32_t>(A->row_ptr), ptr<int32_t>(A->col), ptr<VT>(A->val), x, y,
                      alpha, beta, A->plan.long_thr, alpha == AT(1) && beta == AT(0)};
    a.n_cols = A->n_cols;
    return a;
  }

  template <int S, int R, bool DOT>
  static int csr_launch(const gko_matrix_s* A, const XT* x, XT* y, AT alpha, AT beta, cudaStream_t s,
                        const DotSpec& d, int extra, const int* gate) {
    auto kern = csr_subwarp_kernel<S, R, VT, XT, DOT>;
    static int per_sm = resident_blocks(kern, 256);
    const int64_t rows_per_block = (int64_t)R * (256 / S);
    int64_t g = (A->n_rows + rows_per_block - 1) / rows_per_block;
    int64_t cap = (int64_t)per_sm * sm_count();
    if (DOT && cap > kDotSlots - extra) cap = kDotSlots - extra;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    kern<<<(unsigned)g, 256, 0, s>>>(csr_args(A, x, y, alpha, beta), d, (int)g + extra, gate);
    return (int)g;
  }

  // Row-block launch, CSR or COO (COO: col/val/row from the COO arrays and
  // row blocks from the plan's rb_ptr).
  template <int S, int R, bool DOT, bool COO>
  static int rowblock_launch(const gko_matrix_s* A, const XT* x, XT* y, AT alpha, AT beta, cudaStream_t s,
                             const DotSpec& d, int extra, const int* gate) {
    auto kern = COO ? coo_rowblock_kernel<S, R, VT, XT, DOT> : csr_rowblock_kernel<S, R, VT, XT, DOT>;
    const int cap = A->plan.cap;
    const size_t smem = rb_smem_bytes<VT>(cap, COO);
    // Per device: this kernel's dynamic shared memory limit and its resident
    // blocks per SM by stage size (slot = log2(cap / 512)).  Solves on
    // several host threads (the serving workers) launch concurrently, so the
    // attribute update and the caches change together under one lock.
    struct LaunchCache {
      std::mutex mu;
      size_t smem_allowed[64];
      int per_sm[64][8];
    };
    static LaunchCache lc{};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
      cudaGetLastError();
      fail(GKO_CUDA_ERROR, "row-block kernel: no current device");
      return kLaunchCudaError;
    }
    int slot = 0;
    while ((512 << slot) < cap && slot < 7) ++slot;
    int per_sm = 0;
    {
      std::lock_guard<std::mutex> lk(lc.mu);
      if (lc.smem_allowed[dev] < 48 * 1024) lc.smem_allowed[dev] = 48 * 1024;
      if (smem > lc.smem_allowed[dev]) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
          cudaGetLastError();
          fail(GKO_CUDA_ERROR, "row-block kernel: shared memory request refused");
          return kLaunchCudaError;
        }
        lc.smem_allowed[dev] = smem;
      }
      if (!lc.per_sm[dev][slot]) lc.per_sm[dev][slot] = resident_blocks(kern, kRbThreads, smem);
      per_sm = lc.per_sm[dev][slot];
    }
    constexpr int RB = (kRbThreads / S) * R;
    int64_t g = (A->n_rows + RB - 1) / RB;
    int64_t cap_g = (int64_t)per_sm * sm_count();
    if (DOT && cap_g > kDotSlots - extra) cap_g = kDotSlots - extra;
    if (g > cap_g) g = cap_g;
    if (g < 1) g = 1;
    CsrArgs<VT, XT> ca = csr_args(A, x, y, alpha, beta);
    if (COO) {
      ca.rp = nullptr;
      ca.col = ptr<int32_t>(A->coo_col);
      ca.val = ptr<VT>(A->coo_val);
      ca.row = ptr<int32_t>(A->coo_row);
      ca.rb_ptr = ptr<int32_t>(A->plan.coo_rb);
    }
    const cudaError_t le =
        launch_k(kern, dim3((unsigned)g), dim3(kRbThreads), smem, s, ca, cap, d, (int)g + extra, gate,
                 device_error_word());
    if (le != cudaSuccess) {
      cuda_fail(le, "row-block kernel launch");
      return kLaunchCudaError;
    }
    return (int)g;
  }

  template <bool DOT, bool COO>
  static int rowblock_dispatch(const gko_matrix_s* A, const XT* x, XT* y, AT alpha, AT beta, cudaStream_t s,
                               const DotSpec& d, int extra, const int* gate) {
    const int S = A->plan.S, R = A->plan.R;
#define GKO_RB_CASE(SS, RR) \
  if (S == SS && R == RR) return rowblock_launch<SS, RR, DOT, COO>(A, x, y, alpha, beta, s, d, extra, gate);
#define GKO_RB_ROW(SS) GKO_RB_CASE(SS, 1) GKO_RB_CASE(SS, 2) GKO_RB_CASE(SS, 4)
    GKO_RB_ROW(1) GKO_RB_ROW(2) GKO_RB_ROW(4) GKO_RB_ROW(8)
#undef GKO_RB_ROW
#undef GKO_RB_CASE
    return -1;
  }

  template <bool DOT>
  static int csr_dispatch(const gko_matrix_s* A, const XT* x, XT* y, AT alpha, AT beta, cudaStream_t s,
                          const DotSpec& d, int extra, const int* gate) {
    const int S = A->plan.S, R = A->plan.R;
    if (A->plan.kind == 1) return rowblock_dispatch<DOT, false>(A, x, y, alpha, beta, s, d, extra, gate);
#define GKO_CSR_CASE(SS, RR) \
  if (S == SS && R == RR) return csr_launch<SS, RR, DOT>(A, x, y, alpha, beta, s, d, extra, gate);
#define GKO_CSR_ROW(SS) GKO_CSR_CASE(SS, 1) GKO_CSR_CASE(SS, 2) GKO_CSR_CASE(SS, 4)
    GKO_CSR_ROW(1) GKO_CSR_ROW(2) GKO_CSR_ROW(4) GKO_CSR_ROW(8) GKO_CSR_ROW(16) GKO_CSR_ROW(32)
#undef GKO_CSR_ROW
#undef GKO_CSR_CASE
    return -1;
  }

  static int csr(const gko_matrix_s* A, const XT* x, XT* y, AT alpha, AT beta, cudaStream_t s, void* scratch,
                 const DotSpec* dot, const int* gate) {
    if (A->plan.kind == 3) {  // nonzero split (no fused dot)
      if (A->nnz == 0) {
        scale_kernel<XT, AT><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((A->n_rows + 255) / 256, 4096)),
                               256, 0, s>>>(A->n_rows, y, beta, gate);
        GKO_TRY_CUDA(cudaGetLastError());
        return GKO_OK;
      }
      const int64_t tiles = (A->nnz + kCooTile - 1) / kCooTile;
      AT* carry = static_cast<AT*>(scratch);
      const CsrArgs<VT, XT> ca = csr_args(A, x, y, alpha, beta);
      const int32_t* sr = ptr<int32_t>(A->plan.seg_row);
      if (ca.plain)
        csr_seg_kernel<VT, XT, true><<<(unsigned)tiles, kCooThreads, 0, s>>>(ca, A->nnz, sr, carry, gate);
      else
        csr_seg_kernel<VT, XT, false><<<(unsigned)tiles, kCooThreads, 0, s>>>(ca, A->nnz, sr, carry, gate);
      const unsigned fg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((tiles + 255) / 256, 4096));
      csr_seg_fixup_kernel<VT, XT><<<fg, 256, 0, s>>>(ca, tiles, sr, carry, gate);
      GKO_TRY_CUDA(cudaGetLastError());
      return GKO_OK;
    }
    if (A->plan.kind == 2) {  // merge path (no fused dot)
      const int64_t total = A->n_rows + A->nnz;
      const int64_t tiles = (total + kMergeTile - 1) / kMergeTile;
      AT* carry = static_cast<AT*>(scratch);
      const CsrArgs<VT, XT> ca = csr_args(A, x, y, alpha, beta);
      const int32_t* cx = ptr<int32_t>(A->plan.merge_x);
      csr_merge_kernel<VT, XT><<<(unsigned)tiles, 256, 0, s>>>(ca, A->nnz, cx, carry, gate);
      const unsigned fg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((tiles + 255) / 256, 4096));
      csr_merge_fixup_kernel<VT, XT><<<fg, 256, 0, s>>>(ca, A->nnz, tiles, cx, carry, gate);
      GKO_TRY_CUDA(cudaGetLastError());
      return GKO_OK;
    }
    const bool has_long = A->plan.n_long > 0;
    DotSpec d = dot ? *dot : DotSpec{};
    const int64_t fix_blocks =
        has_long ? std::max<int64_t>(1, std::min<int64_t>((A->plan.n_long + 255) / 256, 256)) : 0;
    const int extra = (int)fix_blocks;
    int g = dot ? csr_dispatch<true>(A, x, y, alpha, beta, s, d, extra, gate)
                : csr_dispatch<false>(A, x, y, alpha, beta, s, d, extra, gate);
    if (g == kLaunchCudaError) return GKO_CUDA_ERROR;
    if (g < 0) return fail(GKO_INVALID_ARG, "unsupported CSR plan");
    if (has_long) {
      AT* partial = static_cast<AT*>(scratch);
      auto kc = csr_long_chunk_kernel<VT, XT>;
      static int per_sm = resident_blocks(kc, 256);
      int64_t blocks = (A->plan.n_chunks + 7) / 8;
      const int64_t cap = (int64_t)per_sm * sm_count();
      if (blocks > cap) blocks = cap;
      if (blocks < 1) blocks = 1;
      kc<<<(unsigned)blocks, 256, 0, s>>>(A->plan.n_chunks, ptr<int32_t>(A->plan.chunk_row),
                                          ptr<int32_t>(A->plan.chunk_start), ptr<int32_t>(A->row_ptr),
                                          ptr<int32_t>(A->col), ptr<VT>(A->val), x, partial, gate);
      const bool plain = alpha == AT(1) && beta == AT(0);
      if (dot)
        csr_long_fixup_kernel<VT, XT, true><<<(unsigned)fix_blocks, 256, 0, s>>>(
            A->plan.n_long, ptr<int32_t>(A->plan.long_rows), ptr<int32_t>(A->plan.long_chunk_ptr), partial, y, alpha,
            beta, plain, d, g, g + extra, gate);
      else
        csr_long_fixup_kernel<VT, XT, false><<<(unsigned)fix_blocks, 256, 0, s>>>(
            A->plan.n_long, ptr<int32_t>(A->plan.long_rows), ptr<int32_t>(A->plan.long_chunk_ptr), partial, y, alpha,
            beta, plain, d, 0, 0, gate);
    }
    GKO_TRY_CUDA(cudaGetLastError());
    return GKO_OK;
  }

  static constexpr int ell_rpt() { return sizeof(VT) == 8 ? 2 : 4; }

  template <bool DOT, bool SELL = false>
  static int ell_launch(const gko_matrix_s* A, const XT* x, XT* y, AT alpha, AT beta, cudaStream_t s,
                        const DotSpec& d, const int* gate) {
    constexpr int RPT = ell_rpt();
    auto kern = ell_kernel<RPT, VT, XT, DOT, SELL>;
    static int per_sm = resident_blocks(kern, 256);
    const int64_t groups = (A->n_rows + RPT - 1) / RPT;
    int64_t g = (groups + 255) / 256;
    int64_t cap = (int64_t)per_sm * sm_count();
    if (DOT && cap > kDotSlots) cap = kDotSlots;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    EllArgs<VT, XT> a{A->n_rows, A->K, A->stride, ptr<int32_t>(A->ell_col), ptr<VT>(A->ell_val), x, y, alpha, beta,
                      alpha == AT(1) && beta == AT(0)};
    if (SELL) {
      a.col = ptr<int32_t>(A->sellp_col);
      a.val = ptr<VT>(A->sellp_val);
      a.C = A->slice;
      while ((1 << a.cshift) < a.C) ++a.cshift;
      a.sets = ptr<int32_t>(A->sellp_sets);
    }
    GKO_TRY_CUDA(launch_k(kern, dim3((unsigned)g), dim3(256), 0, s, a, d, (int)g, gate));
    return GKO_OK;
  }

  static int coo_part(const gko_matrix_s* A, const XT* x, XT* y, AT alpha, AT beta, cudaStream_t s, void* scratch,
                      bool accum, const int* gate) {
    const int64_t nnz = A->coo_nnz;
    if (nnz == 0) {
      if (!accum) {
        scale_kernel<XT, AT><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((A->n_rows + 255) / 256, 4096)),
                               256, 0, s>>>(A->n_rows, y, beta, gate);
        GKO_TRY_CUDA(cudaGetLastError());
      }
      return GKO_OK;
    }
    AT* carry = static_cast<AT*>(scratch);
    CooArgs<VT, XT> a{A->n_rows, A->n_cols, nnz, ptr<int32_t>(A->coo_row), ptr<int32_t>(A->coo_col),
                      ptr<VT>(A->coo_val), x, y, alpha, beta, alpha == AT(1) && beta == AT(0)};
    if (accum)
      coo_launch<VT, XT, true>(a, carry, gate, s);
    else
      coo_launch<VT, XT, false>(a, carry, gate, s);
    GKO_TRY_CUDA(cudaGetLastError());
    return GKO_OK;
  }

  static int run(const gko_matrix_s* A, const XT* x, XT* y, double alpha_d, double beta_d, cudaStream_t s,
                 void* scratch, const DotSpec* dot, const int* gate) {
    const AT alpha = (AT)alpha_d, beta = (AT)beta_d;
    DotSpec d = dot ? *dot : DotSpec{};
    switch (A->fmt) {
      case GKO_CSR:
        return csr(A, x, y, alpha, beta, s, scratch, dot, gate);
      case GKO_ELL:
        return dot ? ell_launch<true>(A, x, y, alpha, beta, s, d, gate)
                   : ell_launch<false>(A, x, y, alpha, beta, s, d, gate);
      case GKO_COO:
        if (A->plan.kind == 1 && A->coo_nnz > 0) {
          const int g = dot ? rowblock_dispatch<true, true>(A, x, y, alpha, beta, s, d, 0, gate)
                            : rowblock_dispatch<false, true>(A, x, y, alpha, beta, s, d, 0, gate);
          if (g == kLaunchCudaError) return GKO_CUDA_ERROR;
          if (g < 0) return fail(GKO_INVALID_ARG, "unsupported COO plan");
          GKO_TRY_CUDA(cudaGetLastError());
          return GKO_OK;
        }
        return coo_part(A, x, y, alpha, beta, s, scratch, false, gate);
      case GKO_SELLP:
        return dot ? ell_launch<true, true>(A, x, y, alpha, beta, s, d, gate)
                   : ell_launch<false, true>(A, x, y, alpha, beta, s, d, gate);
      case GKO_HYBRID:
        GKO_TRY(ell_launch<false>(A, x, y, alpha, beta, s, d, gate));
        return coo_part(A, x, y, alpha, beta, s, scratch, true, gate);
    }
    return fail(GKO_INVALID_ARG, "unknown format");
  }
};

}  // namespace gko
