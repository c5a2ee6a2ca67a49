// Batched CG: many independent small SPD systems solved in one persistent
// launch (the CG of the paper's Section 1 solver list, applied per system).
//
// Layout: the systems' CSR arrays are concatenated (local row pointers, local
// column indices), with per-system row and nonzero offsets.  At creation the
// systems are ordered largest first and grouped into work items: "block"
// items (one system per 256-thread block, vectors r, p, q in shared memory,
// one thread per row, block reductions) for systems above a size threshold,
// and "warp" items (eight systems per block, one per warp, warp-shuffle
// reductions and no block barriers) below it.  Blocks of a persistent grid
// take items from an atomic queue.  The threshold is the tunable: a built-in
// autotuner times the batch with each candidate and keeps the fastest.
// The launch (queue reset + kernel) is captured once into a CUDA graph and
// replayed.  All loops are bounded by the iteration cap; nothing spins.
#include <math.h>

#include <algorithm>
#include <numeric>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "reduce.cuh"

namespace gko {

constexpr int kWarpMaxRows = 256;  // warp mode: rows per system

enum : int { kBRun = 0, kBOk = 1, kBBreak = 2, kBNotConv = 3 };

struct BatchArgs {
  int n_items;
  const int2* items;        // (kind | first << 1, count): kind 0 block, 1 warp
  const int32_t* order;     // systems, largest first
  const int64_t* row_off;   // [count+1]
  const int64_t* nnz_off;   // [count+1]
  const int32_t* rp;        // concatenated local row pointers (n_i + 1 each)
  const int32_t* col;
  const void* val;
  // ELL storage: system i holds ell_k[i] slots per row, slot k of local row r
  // at ell_off[i] + k * n_i + r (column-major within the system), padding
  // column -1
  const int64_t* ell_off;
  const int32_t* ell_k;
  const int32_t* ell_col;
  const void* ell_val;
  // FP32 values of the recurrences of a mixed-precision solve (CSR and ELL
  // order; the stored values themselves for FP32 storage)
  const float* val32;
  const float* ell_val32;
  double delta;       // reliable-update factor
  int32_t* updates;   // per system: reliable updates of the last mixed solve
  const double* b;
  double* x;
  double rel_tol;
  int maxit;
  int32_t* iters;
  double* relres;
  int32_t* status;
  unsigned* queue;
};

// Stored value widened to FP64: FP32 storage goes through the exact integer
// widening (GB300 runs the F2F conversion on its narrow path).
__device__ __forceinline__ double ldv(const double* v, int64_t k) { return v[k]; }
__device__ __forceinline__ double ldv(const float* v, int64_t k) { return widen(v[k]); }

// Sum over a block of THREADS threads, after which one thread derives the
// step's scalars from the total: every thread stores its partial, warp 0
// adds them (lane l the partials l, l + 32, ..., then a 5-step shuffle) and
// its lane 0 runs fin(total, out), writing out[0..3] = red[THREADS ..
// THREADS + 3], which every thread reads after the second barrier.  On
// GB300's narrow FP64 pipe this matters: one warp adds the partials instead
// of every warp running its own shuffle tree, and the divisions and square
// roots of the CG step run once per block, not once per warp.  Barriers: the
// partials are written after every thread passed the previous call's last
// barrier (warp 0 has read the old ones and every thread the old out[]).
template <int THREADS, typename F>
__device__ __forceinline__ const double* block_sum_fin(double v, double* red, F fin) {
  red[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < kWarp) {
    double t = red[threadIdx.x];
#pragma unroll
    for (int j = 1; j < THREADS / kWarp; ++j) t += red[j * kWarp + threadIdx.x];
    t = subwarp_sum<32>(t, 0xffffffffu);
    if (threadIdx.x == 0) fin(t, red + THREADS);
  }
  __syncthreads();
  return red + THREADS;
}

// Row sums of the mixed-precision batched solve: a row's entries in storage
// order (ELL: its slots k*n + i, padding column -1 skipped), four entries'
// column and value loads issued before their FMAs, so each entry's L2
// latency is not exposed in turn (the FP64 solve keeps the plain loop: it is
// FP64-pipe bound, and with FP32 storage the chunked form ran slower there,
// 31.8 -> 40.4 ms).  A: the accumulation type (double for the replaced
// residuals, float for the recurrences).
__device__ __forceinline__ double ldacc(const double* v, int64_t k, double) { return v[k]; }
__device__ __forceinline__ double ldacc(const float* v, int64_t k, double) { return widen(v[k]); }
__device__ __forceinline__ float ldacc(const float* v, int64_t k, float) { return v[k]; }
__device__ __forceinline__ double fmacc(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmacc(float a, float b, float c) { return __fmaf_rn(a, b, c); }

template <typename A, typename VT, typename V>
__device__ __forceinline__ A row_sum_csr(const int32_t* col, const VT* val, int32_t kb, int32_t ke, const V* v) {
  A s = A(0);
  for (int32_t k = kb; k < ke; k += 4) {
    int32_t c[4];
    A w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool ok = k + u < ke;
      c[u] = ok ? col[k + u] : 0;
      w[u] = ok ? ldacc(val, k + u, A(0)) : A(0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (k + u < ke) s = fmacc(w[u], (A)v[c[u]], s);
  }
  return s;
}

template <typename A, typename VT, typename V>
__device__ __forceinline__ A row_sum_ell(const int32_t* col, const VT* val, int K, int n, int i, const V* v) {
  A s = A(0);
  for (int k = 0; k < K; k += 4) {
    int32_t c[4];
    A w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t o = (int64_t)(k + u) * n + i;
      const bool ok = k + u < K;
      c[u] = ok ? col[o] : -1;
      w[u] = ok ? ldacc(val, o, A(0)) : A(0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (c[u] >= 0) s = fmacc(w[u], (A)v[c[u]], s);
  }
  return s;
}

// Group primitives of a solve by G threads (G = THREADS: a block; G = 32: a
// warp): gstep sums v over the group and fin(total, out) derives up to four
// scalars from it (once per block, in every lane of a warp); gsync orders
// the group's shared- and global-memory accesses.
struct Scal {
  double o[4];
};
template <int G, int THREADS, typename F>
__device__ __forceinline__ Scal gstep(double v, double* red, F fin) {
  Scal sc;
  if (G == kWarp) {
    fin(subwarp_sum<32>(v, 0xffffffffu), sc.o);
  } else {
    const double* o = block_sum_fin<THREADS>(v, red, fin);
#pragma unroll
    for (int j = 0; j < 4; ++j) sc.o[j] = o[j];
  }
  return sc;
}
template <int G, int THREADS>
__device__ __forceinline__ double gsum(double v, double* red) {
  return gstep<G, THREADS>(v, red, [](double t, double* o) { o[0] = t; }).o[0];
}
template <int G>
__device__ __forceinline__ void gsync() {
  if (G == kWarp) __syncwarp();
  else __syncthreads();
}

// a / b with a short chain of FP64 operations for the step scalars, which
// one thread computes while its block waits: the hardware reciprocal
// estimate of b refined by two Newton-Raphson steps (r += r (1 - b r), each
// doubling the correct bits) and one correction of the quotient
// (q += r (a - b q)), after Markstein (IBM J. Res. Dev. 34, 1990).  Within an
// ulp or so of the IEEE quotient for normal operands; b must be nonzero and
// finite (the callers divide by a positive p.q or r.r).
// A step flag broadcast as a double (exactly 1.0 or +0.0) tested on its bit
// pattern: an integer compare instead of an FP64 one on the narrow FP64
// pipe, executed by every thread of every iteration.
__device__ __forceinline__ bool flag_on(double f) { return __double_as_longlong(f) != 0; }

__device__ __forceinline__ double quick_div(double a, double b) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(b));
  double e = __fma_rn(-b, r, 1.0);
  r = __fma_rn(r, e, r);
  e = __fma_rn(-b, r, 1.0);
  r = __fma_rn(r, e, r);
  const double q = a * r;
  return __fma_rn(r, __fma_rn(-b, q, a), q);
}

// One CG solve by a group of G threads (G = THREADS: a block; G = 32: a
// warp).  r, p, q: the group's shared-memory vectors.  Follows the
// single-system solver: recurrence residual test, then the true residual; a
// failed true check replaces r and continues.  ELL: the system's entries
// come from its column-major ELL slots (every row's slots in storage order,
// so each row sum is the same sequence of FMAs as from CSR).
template <int G, int THREADS, typename VT, bool ELL>
__device__ void cg_group(const BatchArgs& a, int sys, double* r, double* p, double* q, double* red, int lane) {
  const int64_t r0 = a.row_off[sys];
  const int n = (int)(a.row_off[sys + 1] - r0);
  const int32_t* rp = a.rp + r0 + sys;
  const int64_t k0 = ELL ? a.ell_off[sys] : a.nnz_off[sys];
  const int32_t* col = (ELL ? a.ell_col : a.col) + k0;
  const VT* val = static_cast<const VT*>(ELL ? a.ell_val : a.val) + k0;
  const int K = ELL ? a.ell_k[sys] : 0;
  const double* b = a.b + r0;
  double* x = a.x + r0;
  auto gstep = [&](double v, auto fin) -> Scal { return gko::gstep<G, THREADS>(v, red, fin); };
  auto gsum = [&](double v) -> double { return gko::gsum<G, THREADS>(v, red); };
  auto gsync = [&]() { gko::gsync<G>(); };
  auto row_dot = [&](int i, const double* v) -> double {
    double s = 0.0;
    if (ELL) {
      for (int k = 0; k < K; ++k) {
        const int64_t q = (int64_t)k * n + i;
        const int32_t c = col[q];
        if (c >= 0) s = __fma_rn(ldv(val, q), v[c], s);
      }
    } else {
      for (int32_t k = rp[i]; k < rp[i + 1]; ++k) s = __fma_rn(ldv(val, k), v[col[k]], s);
    }
    return s;
  };
  // r = b - A x0, p = r (x0 staged through q)
  double bb = 0.0;
  for (int i = lane; i < n; i += G) {
    q[i] = x[i];
    bb += b[i] * b[i];
  }
  gsync();
  double rr = 0.0;
  for (int i = lane; i < n; i += G) {
    const double ri = b[i] - row_dot(i, q);
    r[i] = ri;
    p[i] = ri;
    rr += ri * ri;
  }
  const double nb = sqrt(gsum(bb));
  double rho = gsum(rr);
  const double tol = a.rel_tol * nb;
  const double tol2 = tol * tol;  // step tests on squared norms
  int status = kBRun, it = 0;
  double res = nb > 0.0 ? sqrt(rho) / nb : 0.0;
  if (nb == 0.0) {
    for (int i = lane; i < n; i += G) x[i] = 0.0;
    status = kBOk;
  } else if (sqrt(rho) <= tol) {
    status = kBOk;
  }
  gsync();
  while (status == kBRun && it < a.maxit) {
    double pq = 0.0;
    for (int i = lane; i < n; i += G) {
      const double qi = row_dot(i, p);
      q[i] = qi;
      pq += p[i] * qi;
    }
    const Scal sp = gstep(pq, [&](double t, double* o) {
      o[0] = t > 0.0 ? 1.0 : 0.0;
      o[1] = t > 0.0 ? quick_div(rho, t) : 0.0;
    });
    if (!flag_on(sp.o[0])) {
      status = kBBreak;
      break;
    }
    const double alpha = sp.o[1];
    double rn = 0.0;
    for (int i = lane; i < n; i += G) {
      x[i] = __fma_rn(alpha, p[i], x[i]);
      const double ri = __fma_rn(-alpha, q[i], r[i]);
      r[i] = ri;
      rn += ri * ri;
    }
    const Scal sr = gstep(rn, [&](double t, double* o) {
      o[0] = t;
      o[1] = t <= tol2 ? 1.0 : 0.0;
      o[2] = quick_div(t, rho);
    });
    double rho_new = sr.o[0];
    double beta = sr.o[2];
    ++it;
    if (flag_on(sr.o[1])) {
      // true residual b - A x (x staged through q)
      gsync();
      for (int i = lane; i < n; i += G) q[i] = x[i];
      gsync();
      double tt = 0.0;
      for (int i = lane; i < n; i += G) {
        const double ti = b[i] - row_dot(i, q);
        r[i] = ti;
        tt += ti * ti;
      }
      const Scal st = gstep(tt, [&](double t, double* o) {
        o[0] = sqrt(t) / nb;
        o[1] = t <= tol2 ? 1.0 : 0.0;
        o[2] = t;
        o[3] = quick_div(t, rho);
      });
      res = st.o[0];
      if (flag_on(st.o[1])) {
        status = kBOk;
        break;
      }
      rho_new = st.o[2];  // residual replacement
      beta = st.o[3];
    }
    rho = rho_new;
    for (int i = lane; i < n; i += G) p[i] = __fma_rn(beta, p[i], r[i]);
    gsync();
  }
  if (status == kBRun) status = kBNotConv;
  if (status != kBOk) {  // report the true residual of the last iterate
    gsync();
    for (int i = lane; i < n; i += G) q[i] = x[i];
    gsync();
    double tt = 0.0;
    for (int i = lane; i < n; i += G) {
      const double ti = b[i] - row_dot(i, q);
      tt += ti * ti;
    }
    tt = gsum(tt);
    res = nb > 0.0 ? sqrt(tt) / nb : 0.0;
  }
  if (lane == 0) {
    a.iters[sys] = it;
    a.relres[sys] = res;
    a.status[sys] = status;
  }
  gsync();
}

// One mixed-precision CG solve with reliable updates by a group of G threads
// (Sleijpen & van der Vorst 1996; residual replacement without restart,
// van der Vorst & Ye 2000): the recurrences run on the system's FP32 values
// with r, p, q and the iterate's change y in FP32 shared memory, dots and
// scalars in FP64 (FP32 values widened exactly) and each FP64 scalar applied
// as a float pair; when the recurrence residual meets rel_tol ||b|| or drops
// below delta times its largest norm since the last update, y is added to
// the FP64 x, r is replaced by fl32(b - A x) computed in FP64 with the
// system's stored values, and the recurrences go on (rho = r.r of the
// replaced r).  Converged when that FP64 residual meets the tolerance.  Per
// row and iteration this costs two FP64 FMAs (the dots) instead of nnz_i/n_i
// + 5 in the FP64 solve.
template <int G, int THREADS, typename VT, bool ELL>
__device__ void cg_group_rel(const BatchArgs& a, int sys, float* r, float* p, float* q, float* y, double* red,
                             int lane) {
  const int64_t r0 = a.row_off[sys];
  const int n = (int)(a.row_off[sys + 1] - r0);
  const int32_t* rp = a.rp + r0 + sys;
  const int64_t k0 = ELL ? a.ell_off[sys] : a.nnz_off[sys];
  const int32_t* col = (ELL ? a.ell_col : a.col) + k0;
  const VT* val = static_cast<const VT*>(ELL ? a.ell_val : a.val) + k0;
  const float* v32 = (ELL ? a.ell_val32 : a.val32) + k0;
  const int K = ELL ? a.ell_k[sys] : 0;
  const double* b = a.b + r0;
  double* x = a.x + r0;
  // FP64 row product with the stored values over the FP64 x (global memory)
  auto row_dot64 = [&](int i) -> double {
    return ELL ? row_sum_ell<double>(col, val, K, n, i, (const double*)x)
               : row_sum_csr<double>(col, val, rp[i], rp[i + 1], (const double*)x);
  };
  // FP32 row product of the recurrences (FP32 accumulation)
  auto row_dot32 = [&](int i, const float* v) -> float {
    return ELL ? row_sum_ell<float>(col, v32, K, n, i, v) : row_sum_csr<float>(col, v32, rp[i], rp[i + 1], v);
  };
  // r = fl32(b - A x) from the FP64 x; returns ||b - A x||^2 and sets rz = r.r
  auto replace = [&](double& rz) -> double {
    double tt = 0.0, z = 0.0;
    for (int i = lane; i < n; i += G) {
      const double ti = b[i] - row_dot64(i);
      const float tr = __double2float_rn(ti);
      r[i] = tr;
      tt = __fma_rn(ti, ti, tt);
      const double tw = widen(tr);
      z = __fma_rn(tw, tw, z);
    }
    rz = z;
    return tt;
  };
  auto fold = [&]() {  // x += y, y = 0
    gsync<G>();
    for (int i = lane; i < n; i += G) {
      x[i] += widen(y[i]);
      y[i] = 0.0f;
    }
    gsync<G>();
  };
  double bb = 0.0;
  for (int i = lane; i < n; i += G) bb = __fma_rn(b[i], b[i], bb);
  double rz = 0.0;
  const double tt0 = replace(rz);
  for (int i = lane; i < n; i += G) {
    p[i] = r[i];
    y[i] = 0.0f;
  }
  const double nb = sqrt(gsum<G, THREADS>(bb, red));
  const double tn0 = sqrt(gsum<G, THREADS>(tt0, red));
  double rho = gsum<G, THREADS>(rz, red);
  const double tol = a.rel_tol * nb;
  // the step tests compare squared norms (no square root on the critical path)
  const double tol2 = tol * tol, delta2 = a.delta * a.delta;
  double maxrr2 = tn0 * tn0;
  int status = kBRun, it = 0, updates = 0;
  double res = nb > 0.0 ? tn0 / nb : 0.0;
  if (nb == 0.0) {
    for (int i = lane; i < n; i += G) x[i] = 0.0;
    status = kBOk;
  } else if (tn0 <= tol) {
    status = kBOk;
  }
  gsync<G>();
  while (status == kBRun && it < a.maxit) {
    double pq = 0.0;
    for (int i = lane; i < n; i += G) {
      const float qi = row_dot32(i, p);
      q[i] = qi;
      pq = __fma_rn(widen(p[i]), widen(qi), pq);
    }
    const Scal sp = gstep<G, THREADS>(pq, red, [&](double t, double* o) {
      o[0] = t > 0.0 ? 1.0 : 0.0;
      const Lin<float> la(t > 0.0 ? quick_div(rho, t) : 0.0);
      o[1] = la.pack();
      o[2] = Lin<float>(-la.hi, -la.lo).pack();  // the pair of -alpha (exact)
    });
    if (!flag_on(sp.o[0])) {
      status = kBBreak;
      break;
    }
    const Lin<float> ay = Lin<float>::unpack(sp.o[1]), ar = Lin<float>::unpack(sp.o[2]);
    double rn = 0.0;
    for (int i = lane; i < n; i += G) {
      y[i] = ay(p[i], y[i]);
      const float ri = ar(q[i], r[i]);
      r[i] = ri;
      const double rw = widen(ri);
      rn = __fma_rn(rw, rw, rn);
    }
    const Scal sr = gstep<G, THREADS>(rn, red, [&](double t, double* o) {
      const double mx2 = t > maxrr2 ? t : maxrr2;
      o[0] = t;
      o[1] = (t <= tol2 || t < delta2 * mx2) ? 1.0 : 0.0;
      o[2] = Lin<float>(quick_div(t, rho)).pack();
      o[3] = mx2;
    });
    ++it;
    double rho_new = sr.o[0];
    Lin<float> bp = Lin<float>::unpack(sr.o[2]);
    maxrr2 = sr.o[3];
    if (flag_on(sr.o[1])) {  // reliable update
      fold();
      const double tt = replace(rz);
      ++updates;
      const Scal st = gstep<G, THREADS>(tt, red, [&](double t, double* o) {
        o[0] = sqrt(t) / nb;
        o[1] = t <= tol2 ? 1.0 : 0.0;
        o[2] = t;
      });
      res = st.o[0];
      if (flag_on(st.o[1])) {
        status = kBOk;
        break;
      }
      maxrr2 = st.o[2];
      const Scal sz = gstep<G, THREADS>(rz, red, [&](double t, double* o) {
        o[0] = t;
        o[1] = Lin<float>(quick_div(t, rho)).pack();
      });
      rho_new = sz.o[0];
      bp = Lin<float>::unpack(sz.o[1]);
    }
    rho = rho_new;
    for (int i = lane; i < n; i += G) p[i] = bp(p[i], r[i]);
    gsync<G>();
  }
  if (status == kBRun) status = kBNotConv;
  if (status != kBOk) {  // fold what moved since the last update; report the true residual
    fold();
    double tt = 0.0;
    for (int i = lane; i < n; i += G) {
      const double ti = b[i] - row_dot64(i);
      tt = __fma_rn(ti, ti, tt);
    }
    tt = gsum<G, THREADS>(tt, red);
    res = nb > 0.0 ? sqrt(tt) / nb : 0.0;
  }
  if (lane == 0) {
    a.iters[sys] = it;
    a.relres[sys] = res;
    a.status[sys] = status;
    a.updates[sys] = updates;
  }
  gsync<G>();
}

// The mixed-precision counterpart of batch_cg_kernel: the same persistent
// schedule, with four FP32 vectors (r, p, q, y) per system in shared memory.
template <int THREADS, typename VT, bool ELL>
__global__ void __launch_bounds__(THREADS) batch_cg_rel_kernel(BatchArgs a, int block_rows) {
  extern __shared__ __align__(16) float smf[];
  __shared__ double red[THREADS + 4];
  __shared__ int item_s;
  for (;;) {
    if (threadIdx.x == 0) item_s = (int)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int item = item_s;
    __syncthreads();
    if (item >= a.n_items) return;
    const int2 it = a.items[item];
    const int kind = it.x & 1, first = it.x >> 1;
    if (kind == 0) {
      float* v = smf;
      cg_group_rel<THREADS, THREADS, VT, ELL>(a, a.order[first], v, v + block_rows, v + 2 * block_rows,
                                              v + 3 * block_rows, red, threadIdx.x);
    } else {
      const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
      float* base = smf + (size_t)w * 4 * kWarpMaxRows;
      if (w < it.y)
        cg_group_rel<kWarp, THREADS, VT, ELL>(a, a.order[first + w], base, base + kWarpMaxRows,
                                              base + 2 * kWarpMaxRows, base + 3 * kWarpMaxRows, red, lane);
      __syncthreads();
    }
  }
}

// Persistent batched CG: blocks of THREADS threads take work items from an
// atomic queue, largest systems first; a block item is one system solved by
// the whole block, a warp item THREADS/32 systems, one per warp.
template <int THREADS, typename VT, bool ELL>
__global__ void __launch_bounds__(THREADS) batch_cg_kernel(BatchArgs a, int block_rows) {
  extern __shared__ __align__(16) double sm[];
  __shared__ double red[THREADS + 4];  // partials + the step's scalars
  __shared__ int item_s;
  for (;;) {
    if (threadIdx.x == 0) item_s = (int)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int item = item_s;
    __syncthreads();
    if (item >= a.n_items) return;
    const int2 it = a.items[item];
    const int kind = it.x & 1, first = it.x >> 1;
    if (kind == 0) {
      double* r = sm;
      double* p = sm + block_rows;
      double* q = sm + 2 * block_rows;
      cg_group<THREADS, THREADS, VT, ELL>(a, a.order[first], r, p, q, red, threadIdx.x);
    } else {
      const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
      double* base = sm + (size_t)w * 3 * kWarpMaxRows;
      if (w < it.y)
        cg_group<kWarp, THREADS, VT, ELL>(a, a.order[first + w], base, base + kWarpMaxRows, base + 2 * kWarpMaxRows,
                                          red, lane);
      __syncthreads();
    }
  }
}

// FP64 -> FP32 rounding (to nearest even) of the systems' values for FP32
// storage; the same rounding as gko_matrix_convert_values.
__global__ void round_f32_kernel(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __double2float_rn(a[i]);
}

}  // namespace gko

using namespace gko;

struct gko_batch_s {
  int32_t count = 0;
  gko_dtype dtype = GKO_F64;
  int64_t total_rows = 0, total_nnz = 0;
  int32_t max_rows = 0;
  Buf row_off, nnz_off, rp, col, val, order, items, iters, relres, status, queue;
  Buf ell_off, ell_k, ell_col, ell_val;  // the same systems in per-system column-major ELL
  int64_t ell_slots = 0;
  // mixed precision (reliable updates): FP32 values of the recurrences (the
  // stored ones for FP32 storage) and per-system update counts
  int32_t mixed = 0;
  double delta = 0.1;
  Buf val32, ell_val32, updates;
  std::vector<int64_t> h_rows;   // rows per system
  std::vector<int32_t> h_order;  // largest first
  int32_t threshold = 0;         // warp mode for systems with <= threshold rows
  int32_t threads = 256;         // threads per block (a block item's group size)
  int32_t ell = 0;               // 1: solve from the ELL arrays
  int n_items = 0;
  int block_rows = 0;
  // cached graph of (queue reset + kernel)
  cudaGraphExec_t exec = nullptr;
  const double* g_b = nullptr;
  double* g_x = nullptr;
  double g_tol = -1;
  int g_maxit = -1;
  cudaStream_t g_stream = nullptr;
  ~gko_batch_s() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

namespace gko {

static int build_items(gko_batch B, int32_t threshold, cudaStream_t s) {
  threshold = std::min(threshold, kWarpMaxRows);
  std::vector<int2> items;
  int block_rows = 0;
  size_t i = 0;
  const size_t n = B->h_order.size();
  while (i < n && B->h_rows[B->h_order[i]] > threshold) {
    block_rows = std::max<int>(block_rows, (int)B->h_rows[B->h_order[i]]);
    items.push_back(make_int2((int)(i << 1) | 0, 1));
    ++i;
  }
  const size_t per_item = (size_t)B->threads / kWarp;
  while (i < n) {
    const int cnt = (int)std::min<size_t>(per_item, n - i);
    items.push_back(make_int2((int)(i << 1) | 1, cnt));
    i += cnt;
  }
  GKO_TRY(alloc(sizeof(int2) * std::max<size_t>(1, items.size()), &B->items));
  if (!items.empty())
    GKO_TRY_CUDA(cudaMemcpyAsync(B->items->ptr, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, s));
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  B->threshold = threshold;
  B->n_items = (int)items.size();
  B->block_rows = block_rows;
  if (B->exec) {
    cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
  }
  return GKO_OK;
}

static size_t batch_smem(const gko_batch_s* B) {
  // FP64: r, p, q as doubles; mixed: r, p, q, y as floats
  const size_t per = B->mixed ? 4 * sizeof(float) : 3 * sizeof(double);
  const size_t blk = per * B->block_rows;
  const size_t wrp = B->threshold > 0 ? (size_t)(B->threads / kWarp) * per * kWarpMaxRows : 0;
  return std::max<size_t>(std::max(blk, wrp), 16);
}

template <int T, typename VT, bool E>
static int batch_launch_t(const BatchArgs& a, int n_items, int block_rows, size_t smem, bool mixed, cudaStream_t s) {
  auto kern = mixed ? batch_cg_rel_kernel<T, VT, E> : batch_cg_kernel<T, VT, E>;
  GKO_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 1;
  GKO_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem));
  const int grid = std::max(1, std::min(n_items, std::max(1, per_sm) * sm_count()));
  kern<<<grid, T, smem, s>>>(a, block_rows);
  GKO_TRY_CUDA(cudaGetLastError());
  return GKO_OK;
}

static int batch_launch(gko_batch B, const double* b, double* x, double tol, int maxit, cudaStream_t s) {
  BatchArgs a;
  a.n_items = B->n_items;
  a.items = ptr<int2>(B->items);
  a.order = ptr<int32_t>(B->order);
  a.row_off = ptr<int64_t>(B->row_off);
  a.nnz_off = ptr<int64_t>(B->nnz_off);
  a.rp = ptr<int32_t>(B->rp);
  a.col = ptr<int32_t>(B->col);
  a.val = B->val->ptr;
  a.b = b;
  a.x = x;
  a.rel_tol = tol;
  a.maxit = maxit;
  a.iters = ptr<int32_t>(B->iters);
  a.relres = ptr<double>(B->relres);
  a.status = ptr<int32_t>(B->status);
  a.queue = ptr<unsigned>(B->queue);
  a.ell_off = ptr<int64_t>(B->ell_off);
  a.ell_k = ptr<int32_t>(B->ell_k);
  a.ell_col = ptr<int32_t>(B->ell_col);
  a.ell_val = B->ell_val ? B->ell_val->ptr : nullptr;
  a.val32 = B->val32 ? ptr<float>(B->val32) : nullptr;
  a.ell_val32 = B->ell_val32 ? ptr<float>(B->ell_val32) : nullptr;
  a.delta = B->delta;
  a.updates = ptr<int32_t>(B->updates);
  const size_t smem = batch_smem(B);
  GKO_TRY_CUDA(cudaMemsetAsync(B->queue->ptr, 0, sizeof(unsigned), s));
  if (!B->mixed) GKO_TRY_CUDA(cudaMemsetAsync(B->updates->ptr, 0, sizeof(int32_t) * B->count, s));
  const bool f64 = B->dtype == GKO_F64;
  switch (B->threads * 4 + (f64 ? 2 : 0) + (B->ell ? 1 : 0)) {
#define GKO_BATCH_CASE(T, VT, E) \
  case T * 4 + (std::is_same<VT, double>::value ? 2 : 0) + (E ? 1 : 0): \
    return batch_launch_t<T, VT, E>(a, B->n_items, B->block_rows, smem, B->mixed != 0, s);
#define GKO_BATCH_T(T) \
  GKO_BATCH_CASE(T, double, false) GKO_BATCH_CASE(T, double, true) GKO_BATCH_CASE(T, float, false) \
  GKO_BATCH_CASE(T, float, true)
    GKO_BATCH_T(256) GKO_BATCH_T(512) GKO_BATCH_T(1024)
#undef GKO_BATCH_T
#undef GKO_BATCH_CASE
  }
  return fail(GKO_INVALID_ARG, "unsupported batch schedule");
}

// Capture (queue reset + kernel) once per (b, x, tol, maxit, stream) and
// replay it afterwards.
static int batch_run(gko_batch B, const double* b, double* x, double tol, int maxit, cudaStream_t s) {
  const bool same = B->exec && B->g_b == b && B->g_x == x && B->g_tol == tol && B->g_maxit == maxit &&
                    B->g_stream == s;
  if (!same) {
    if (B->exec) {
      cudaGraphExecDestroy(B->exec);
      B->exec = nullptr;
    }
    cudaStream_t cs;
    GKO_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph;
    GKO_TRY_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const int st = batch_launch(B, b, x, tol, maxit, cs);
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (st != GKO_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&B->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      B->exec = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    B->g_b = b;
    B->g_x = x;
    B->g_tol = tol;
    B->g_maxit = maxit;
    B->g_stream = s;
  }
  GKO_TRY_CUDA(cudaGraphLaunch(B->exec, s));
  return GKO_OK;
}

// The systems in per-system column-major ELL (the batch's ELL storage):
// system i keeps K_i = its longest row slots per row, slot k of local row r
// at ell_off[i] + k * n_i + r, filled from the CSR rows in storage order,
// padding column -1 and value 0.  Values FP64, rounded to FP32 on the device
// for FP32 storage (the rounding of gko_batch_create).
static int build_ell(gko_batch B, const int64_t* row_off, const int64_t* nnz_off, const int32_t* row_ptr,
                     const int32_t* col, const double* values, cudaStream_t s) {
  const int32_t count = B->count;
  std::vector<int64_t> off((size_t)count + 1, 0);
  std::vector<int32_t> kk((size_t)count, 0);
  for (int32_t i = 0; i < count; ++i) {
    const int64_t n = row_off[i + 1] - row_off[i];
    const int32_t* rp = row_ptr + row_off[i] + i;
    int32_t k = 0;
    for (int64_t r = 0; r < n; ++r) k = std::max(k, rp[r + 1] - rp[r]);
    kk[(size_t)i] = k;
    off[(size_t)i + 1] = off[(size_t)i] + (int64_t)k * n;
  }
  const int64_t slots = off[(size_t)count];
  std::vector<int32_t> ecol((size_t)std::max<int64_t>(slots, 1), -1);
  std::vector<double> eval((size_t)std::max<int64_t>(slots, 1), 0.0);
  for (int32_t i = 0; i < count; ++i) {
    const int64_t n = row_off[i + 1] - row_off[i];
    const int32_t* rp = row_ptr + row_off[i] + i;
    const int64_t k0 = nnz_off[i];
    for (int64_t r = 0; r < n; ++r)
      for (int32_t k = rp[r]; k < rp[r + 1]; ++k) {
        const int64_t q = off[(size_t)i] + (int64_t)(k - rp[r]) * n + r;
        ecol[(size_t)q] = col[k0 + k];
        eval[(size_t)q] = values[k0 + k];
      }
  }
  const size_t vs = dtype_size(B->dtype);
  GKO_TRY(alloc(sizeof(int64_t) * (count + 1), &B->ell_off));
  GKO_TRY(alloc(sizeof(int32_t) * count, &B->ell_k));
  GKO_TRY(alloc(sizeof(int32_t) * std::max<int64_t>(slots, 1), &B->ell_col));
  GKO_TRY(alloc(vs * std::max<int64_t>(slots, 1), &B->ell_val));
  GKO_TRY_CUDA(cudaMemcpyAsync(B->ell_off->ptr, off.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s));
  GKO_TRY_CUDA(cudaMemcpyAsync(B->ell_k->ptr, kk.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, s));
  if (slots > 0) {
    GKO_TRY_CUDA(cudaMemcpyAsync(B->ell_col->ptr, ecol.data(), sizeof(int32_t) * slots, cudaMemcpyHostToDevice, s));
    if (B->dtype == GKO_F64) {
      GKO_TRY_CUDA(cudaMemcpyAsync(B->ell_val->ptr, eval.data(), sizeof(double) * slots, cudaMemcpyHostToDevice, s));
    } else {
      Scratch v64;
      GKO_TRY(v64.get(sizeof(double) * slots, s));
      GKO_TRY_CUDA(cudaMemcpyAsync(v64.data(), eval.data(), sizeof(double) * slots, cudaMemcpyHostToDevice, s));
      round_f32_kernel<<<(unsigned)std::min<int64_t>((slots + 255) / 256, (int64_t)sm_count() * 16), 256, 0, s>>>(
          slots, v64.as<double>(), ptr<float>(B->ell_val));
      GKO_TRY_CUDA(cudaGetLastError());
      GKO_TRY_CUDA(cudaStreamSynchronize(s));
    }
  }
  GKO_TRY_CUDA(cudaStreamSynchronize(s));  // the host arrays above go out of scope
  B->ell_slots = slots;
  return GKO_OK;
}

}  // namespace gko

extern "C" {

int gko_batch_create(int32_t count, const int64_t* row_off, const int64_t* nnz_off, const int32_t* row_ptr,
                     const int32_t* col, const double* values, gko_dtype storage, void* stream, gko_batch* out) {
  if (!out) return fail(GKO_INVALID_ARG, "null out");
  *out = nullptr;
  if (count <= 0 || !row_off || !nnz_off || !row_ptr || !col || !values)
    return fail(GKO_INVALID_ARG, "bad batch arguments");
  if (storage != GKO_F64 && storage != GKO_F32) return fail(GKO_INVALID_ARG, "batch storage must be F64 or F32");
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<gko_batch_s> B(new gko_batch_s());
  B->count = count;
  B->dtype = storage;
  B->total_rows = row_off[count];
  B->total_nnz = nnz_off[count];
  if (row_off[0] != 0 || nnz_off[0] != 0 || B->total_nnz >= INT32_MAX)
    return fail(GKO_INVALID_ARG, "offsets must start at 0 and nnz fit int32");
  B->h_rows.resize(count);
  for (int32_t i = 0; i < count; ++i) {
    const int64_t n = row_off[i + 1] - row_off[i], z = nnz_off[i + 1] - nnz_off[i];
    if (n <= 0 || z < 0) return fail(GKO_INVALID_ARG, "every system needs rows");
    const int32_t* rp = row_ptr + row_off[i] + i;
    if (rp[0] != 0 || rp[n] != z) return fail(GKO_INVALID_ARG, "system row pointers must run 0..nnz_i");
    for (int64_t r = 0; r < n; ++r)
      if (rp[r] > rp[r + 1]) return fail(GKO_INVALID_ARG, "row pointers must not decrease");
    for (int64_t k = nnz_off[i]; k < nnz_off[i + 1]; ++k)
      if (col[k] < 0 || col[k] >= n) return fail(GKO_INVALID_ARG, "column index out of range");
    B->h_rows[i] = n;
    B->max_rows = std::max<int32_t>(B->max_rows, (int32_t)n);
  }
  if (B->max_rows > 8192) return fail(GKO_NOT_SUPPORTED, "batched systems are limited to 8192 rows");
  B->h_order.resize(count);
  std::iota(B->h_order.begin(), B->h_order.end(), 0);
  std::stable_sort(B->h_order.begin(), B->h_order.end(),
                   [&](int32_t a, int32_t b) { return B->h_rows[a] > B->h_rows[b]; });
  const int64_t nrp = B->total_rows + count;
  const size_t vs = dtype_size(storage);
  GKO_TRY(alloc(sizeof(int64_t) * (count + 1), &B->row_off));
  GKO_TRY(alloc(sizeof(int64_t) * (count + 1), &B->nnz_off));
  GKO_TRY(alloc(sizeof(int32_t) * nrp, &B->rp));
  GKO_TRY(alloc(sizeof(int32_t) * B->total_nnz, &B->col));
  GKO_TRY(alloc(vs * B->total_nnz, &B->val));
  GKO_TRY(alloc(sizeof(int32_t) * count, &B->order));
  GKO_TRY(alloc(sizeof(int32_t) * count, &B->iters));
  GKO_TRY(alloc(sizeof(double) * count, &B->relres));
  GKO_TRY(alloc(sizeof(int32_t) * count, &B->status));
  GKO_TRY(alloc(sizeof(int32_t) * count, &B->updates));
  GKO_TRY_CUDA(cudaMemsetAsync(B->updates->ptr, 0, sizeof(int32_t) * count, s));
  GKO_TRY(alloc(sizeof(unsigned), &B->queue));
  GKO_TRY_CUDA(cudaMemcpyAsync(B->row_off->ptr, row_off, sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s));
  GKO_TRY_CUDA(cudaMemcpyAsync(B->nnz_off->ptr, nnz_off, sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s));
  GKO_TRY_CUDA(cudaMemcpyAsync(B->rp->ptr, row_ptr, sizeof(int32_t) * nrp, cudaMemcpyHostToDevice, s));
  GKO_TRY_CUDA(cudaMemcpyAsync(B->col->ptr, col, sizeof(int32_t) * B->total_nnz, cudaMemcpyHostToDevice, s));
  if (storage == GKO_F64) {
    GKO_TRY_CUDA(cudaMemcpyAsync(B->val->ptr, values, sizeof(double) * B->total_nnz, cudaMemcpyHostToDevice, s));
  } else if (B->total_nnz > 0) {
    // FP32 storage: the FP64 values are rounded to nearest on the device
    Scratch v64;
    GKO_TRY(v64.get(sizeof(double) * B->total_nnz, s));
    GKO_TRY_CUDA(cudaMemcpyAsync(v64.data(), values, sizeof(double) * B->total_nnz, cudaMemcpyHostToDevice, s));
    round_f32_kernel<<<(unsigned)std::min<int64_t>((B->total_nnz + 255) / 256, (int64_t)sm_count() * 16), 256, 0,
                       s>>>(B->total_nnz, v64.as<double>(), ptr<float>(B->val));
    GKO_TRY_CUDA(cudaGetLastError());
    GKO_TRY_CUDA(cudaStreamSynchronize(s));
  }
  GKO_TRY_CUDA(cudaMemcpyAsync(B->order->ptr, B->h_order.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, s));
  GKO_TRY(build_ell(B.get(), row_off, nnz_off, row_ptr, col, values, s));
  GKO_TRY(build_items(B.get(), 144, s));
  *out = B.release();
  return GKO_OK;
}

int gko_batch_create_systems(int32_t count, const int32_t* n_rows, const int32_t* const* row_ptrs,
                             const int32_t* const* cols, const double* const* values, gko_dtype storage, void* stream,
                             gko_batch* out) {
  if (!out) return fail(GKO_INVALID_ARG, "null out");
  *out = nullptr;
  if (count <= 0 || !n_rows || !row_ptrs || !cols || !values) return fail(GKO_INVALID_ARG, "bad batch arguments");
  // offsets from the systems' sizes, then the concatenated arrays (checked
  // in full by gko_batch_create)
  std::vector<int64_t> row_off((size_t)count + 1, 0), nnz_off((size_t)count + 1, 0);
  for (int32_t i = 0; i < count; ++i) {
    if (n_rows[i] <= 0 || !row_ptrs[i]) return fail(GKO_INVALID_ARG, "every system needs rows and row pointers");
    const int64_t z = row_ptrs[i][n_rows[i]];
    if (z < 0 || (z > 0 && (!cols[i] || !values[i]))) return fail(GKO_INVALID_ARG, "bad system arrays");
    row_off[i + 1] = row_off[i] + n_rows[i];
    nnz_off[i + 1] = nnz_off[i] + z;
    if (nnz_off[i + 1] >= INT32_MAX) return fail(GKO_INVALID_ARG, "the batch's nonzeros must fit int32");
  }
  std::vector<int32_t> rp((size_t)(row_off[count] + count)), col((size_t)nnz_off[count]);
  std::vector<double> val((size_t)nnz_off[count]);
  for (int32_t i = 0; i < count; ++i) {
    std::copy(row_ptrs[i], row_ptrs[i] + n_rows[i] + 1, rp.begin() + (row_off[i] + i));
    const int64_t z = nnz_off[i + 1] - nnz_off[i];
    if (z > 0) {
      std::copy(cols[i], cols[i] + z, col.begin() + nnz_off[i]);
      std::copy(values[i], values[i] + z, val.begin() + nnz_off[i]);
    }
  }
  const int st = gko_batch_create(count, row_off.data(), nnz_off.data(), rp.data(), col.data(), val.data(), storage,
                                  stream, out);
  // the pageable sources above must outlive the copies gko_batch_create enqueued
  if (st == GKO_OK) GKO_TRY_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return st;
}

int gko_batch_export(gko_batch B, int64_t* row_off, int64_t* nnz_off, int32_t* row_ptr, int32_t* col, void* values,
                     void* stream) {
  if (!B) return fail(GKO_INVALID_ARG, "null batch");
  cudaStream_t s = (cudaStream_t)stream;
  auto get = [&](void* dst, const Buf& b, size_t bytes) -> int {
    if (dst && b && bytes) GKO_TRY_CUDA(cudaMemcpyAsync(dst, b->ptr, bytes, cudaMemcpyDeviceToHost, s));
    return GKO_OK;
  };
  GKO_TRY(get(row_off, B->row_off, sizeof(int64_t) * (B->count + 1)));
  GKO_TRY(get(nnz_off, B->nnz_off, sizeof(int64_t) * (B->count + 1)));
  GKO_TRY(get(row_ptr, B->rp, sizeof(int32_t) * (B->total_rows + B->count)));
  GKO_TRY(get(col, B->col, sizeof(int32_t) * B->total_nnz));
  GKO_TRY(get(values, B->val, dtype_size(B->dtype) * B->total_nnz));
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  return GKO_OK;
}

int gko_batch_set_threshold(gko_batch B, int32_t warp_rows, void* stream) {
  if (!B || warp_rows < 0) return fail(GKO_INVALID_ARG, "bad batch threshold");
  return build_items(B, warp_rows, (cudaStream_t)stream);
}

int gko_batch_set_schedule(gko_batch B, int32_t warp_rows, int32_t threads, int32_t storage, void* stream) {
  if (!B || warp_rows < 0 || (threads != 256 && threads != 512 && threads != 1024) ||
      (storage != GKO_BATCH_CSR && storage != GKO_BATCH_ELL))
    return fail(GKO_INVALID_ARG, "batch schedule: warp_rows >= 0, threads 256/512/1024, storage CSR or ELL");
  B->threads = threads;
  B->ell = storage == GKO_BATCH_ELL ? 1 : 0;
  return build_items(B, warp_rows, (cudaStream_t)stream);
}

int gko_batch_set_precision(gko_batch B, int32_t precision, double reliable_delta, void* stream) {
  if (!B || (precision != GKO_PRECISION_F64 && precision != GKO_PRECISION_MIXED_F32) ||
      !(reliable_delta >= 0.0 && reliable_delta < 1.0))
    return fail(GKO_INVALID_ARG, "batch precision: F64 or MIXED_F32, reliable_delta in [0, 1)");
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == GKO_PRECISION_MIXED_F32 && !B->val32) {
    if (B->dtype == GKO_F32) {  // the stored values are the recurrences' values
      B->val32 = B->val;
      B->ell_val32 = B->ell_val;
    } else {
      Buf v, e;
      GKO_TRY(alloc(sizeof(float) * std::max<int64_t>(B->total_nnz, 1), &v));
      GKO_TRY(alloc(sizeof(float) * std::max<int64_t>(B->ell_slots, 1), &e));
      const int g = sm_count() * 16;
      if (B->total_nnz > 0)
        round_f32_kernel<<<(unsigned)std::min<int64_t>((B->total_nnz + 255) / 256, g), 256, 0, s>>>(
            B->total_nnz, ptr<double>(B->val), ptr<float>(v));
      if (B->ell_slots > 0)
        round_f32_kernel<<<(unsigned)std::min<int64_t>((B->ell_slots + 255) / 256, g), 256, 0, s>>>(
            B->ell_slots, ptr<double>(B->ell_val), ptr<float>(e));
      GKO_TRY_CUDA(cudaGetLastError());
      GKO_TRY_CUDA(cudaStreamSynchronize(s));
      B->val32 = v;
      B->ell_val32 = e;
    }
  }
  B->mixed = precision == GKO_PRECISION_MIXED_F32 ? 1 : 0;
  B->delta = reliable_delta > 0.0 ? reliable_delta : 0.1;
  if (B->exec) {
    cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
  }
  return GKO_OK;
}

int gko_batch_last_updates(gko_batch B, int32_t* updates, void* stream) {
  if (!B || !updates) return fail(GKO_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  GKO_TRY_CUDA(cudaMemcpyAsync(updates, B->updates->ptr, sizeof(int32_t) * B->count, cudaMemcpyDeviceToHost, s));
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  return GKO_OK;
}

int gko_batch_info(gko_batch B, int32_t* count, int64_t* total_rows, int64_t* total_nnz, int32_t* warp_rows,
                   int32_t* n_items, int32_t* threads, int32_t* storage) {
  if (!B) return fail(GKO_INVALID_ARG, "null batch");
  if (count) *count = B->count;
  if (total_rows) *total_rows = B->total_rows;
  if (total_nnz) *total_nnz = B->total_nnz;
  if (warp_rows) *warp_rows = B->threshold;
  if (n_items) *n_items = B->n_items;
  if (threads) *threads = B->threads;
  if (storage) *storage = B->ell ? GKO_BATCH_ELL : GKO_BATCH_CSR;
  return GKO_OK;
}

int gko_batch_cg(gko_batch B, const double* b, double* x, double rel_tol, int32_t max_iters, int32_t* iterations,
                 double* rel_residuals, int32_t* statuses, void* stream) {
  if (!B || !b || !x || !(rel_tol >= 0.0) || max_iters < 0) return fail(GKO_INVALID_ARG, "bad batch solve arguments");
  cudaStream_t s = (cudaStream_t)stream;
  GKO_TRY(batch_run(B, b, x, rel_tol, max_iters, s));
  if (iterations)
    GKO_TRY_CUDA(cudaMemcpyAsync(iterations, B->iters->ptr, sizeof(int32_t) * B->count, cudaMemcpyDeviceToHost, s));
  if (rel_residuals)
    GKO_TRY_CUDA(
        cudaMemcpyAsync(rel_residuals, B->relres->ptr, sizeof(double) * B->count, cudaMemcpyDeviceToHost, s));
  std::vector<int32_t> st(B->count);
  GKO_TRY_CUDA(cudaMemcpyAsync(st.data(), B->status->ptr, sizeof(int32_t) * B->count, cudaMemcpyDeviceToHost, s));
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  int worst = GKO_OK;
  for (int32_t i = 0; i < B->count; ++i) {
    const int code = st[i] == kBOk ? GKO_OK : st[i] == kBBreak ? GKO_BREAKDOWN : GKO_NOT_CONVERGED;
    if (statuses) statuses[i] = code;
    if (code == GKO_BREAKDOWN || (code == GKO_NOT_CONVERGED && worst == GKO_OK)) worst = code;
  }
  return worst;
}

// Autotuner: time the whole batch for every schedule (warp-mode threshold x
// threads per block x storage) on a scratch copy of x0 and keep the fastest.
int gko_batch_tune(gko_batch B, const double* b, const double* x0, double rel_tol, int32_t max_iters,
                   int32_t* warp_rows, int32_t* threads, int32_t* storage, float* best_ms, void* stream) {
  if (!B || !b || !x0) return fail(GKO_INVALID_ARG, "bad tune arguments");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch xs;
  GKO_TRY(xs.get(sizeof(double) * B->total_rows, s));
  struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  GKO_TRY_CUDA(cudaEventCreate(&ev.a));
  GKO_TRY_CUDA(cudaEventCreate(&ev.b));
  float best = 1e30f;
  int32_t best_t = B->threshold, best_th = B->threads, best_st = B->ell ? GKO_BATCH_ELL : GKO_BATCH_CSR;
  for (int32_t st : {GKO_BATCH_CSR, GKO_BATCH_ELL})
    for (int32_t th : {256, 512, 1024})
      for (int32_t t : {0, 64, 144, 256}) {
        GKO_TRY(gko_batch_set_schedule(B, t, th, st, stream));
        for (int rep = 0; rep < 2; ++rep) {
          GKO_TRY_CUDA(cudaMemcpyAsync(xs.data(), x0, sizeof(double) * B->total_rows, cudaMemcpyDeviceToDevice, s));
          GKO_TRY_CUDA(cudaEventRecord(ev.a, s));
          GKO_TRY(batch_run(B, b, xs.as<double>(), rel_tol, max_iters, s));
          GKO_TRY_CUDA(cudaEventRecord(ev.b, s));
          GKO_TRY_CUDA(cudaEventSynchronize(ev.b));
          float ms = 0.f;
          GKO_TRY_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
          if (rep == 1 && ms < best) {
            best = ms;
            best_t = t;
            best_th = th;
            best_st = st;
          }
        }
      }
  GKO_TRY(gko_batch_set_schedule(B, best_t, best_th, best_st, stream));
  if (warp_rows) *warp_rows = best_t;
  if (threads) *threads = best_th;
  if (storage) *storage = best_st;
  if (best_ms) *best_ms = best;
  return GKO_OK;
}

int gko_batch_destroy(gko_batch B) {
  delete B;
  return GKO_OK;
}

}  // extern "C"
