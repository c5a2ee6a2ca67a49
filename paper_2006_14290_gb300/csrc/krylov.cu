// Krylov solvers on the device: CG, BiCGSTAB and restarted GMRES (the solver
// family the paper's Section 1 lists and Section 4 times), and
// mixed-precision iterative refinement around them.
//
// Design: every vector kernel that ends in a reduction finishes with the
// "last block" pattern of reduce.cuh, and that block's thread 0 runs the
// scalar step of the method (alpha, beta, omega, convergence and breakdown
// tests, iteration count) on the device state `Ctl`.  Every kernel of an
// iteration is gated by Ctl::done, so the host enqueues batches of iterations
// and only polls the state every few iterations; iterations enqueued after
// convergence cost one empty launch each.  Dots and norms accumulate in FP64;
// vectors are stored as T (double, or float for the inner solve of mixed
// precision) with every update computed in FP64 and rounded once on store.
#include <cooperative_groups.h>
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "blas1.cuh"
#include "reduce.cuh"
#include "spmv.cuh"
#include "precond.cuh"

namespace gko {

enum : int { kRun = 0, kConverged = 1, kBreakdown = 2, kNotConverged = 3, kCheck = 4 };

// Device-resident solver state.  The first three ints are gate words: an
// SpMV gated on &done runs unless done|zero; gated on &phase it also stops
// when `phase` is set (BiCGSTAB half step converged / GMRES cycle ended).
struct Ctl {
  int phase;
  int done;
  int zero;
  int status;
  int iter;
  int maxit;
  int replace;
  int check_true;
  int cycles;
  int k;         // GMRES: columns of the finished cycle
  int noreorth;  // GMRES: this step skips the second Gram-Schmidt pass
  int pad;
  double nb, tol_abs;
  double rho, rho_new, alpha, beta, omega;
  double red[4];  // fused SpMV dots: red[0] = w.y, red[1] = y.y
  double rr;
  // reliable updates (mixed precision): an update is due when the recurrence
  // residual drops below delta times maxrr, its largest norm since the last
  // update (delta = 0: only at convergence); half: the last check came from
  // BiCGSTAB's half step
  double maxrr, delta;
  int half;
  int pad2;
};

__device__ __forceinline__ double wd(double v) { return v; }
__device__ __forceinline__ double wd(float v) { return widen(v); }

__device__ __forceinline__ double dsq(double a) { return a * a; }

template <typename T>
struct LinPair {
  Lin<T> a, b;
};
template <typename T>
struct LinTriple {
  Lin<T> a, b, c;
};

// One value per block: thread 0 evaluates f() and the block reads it from
// shared memory.  The step scalars need an FP64 division and, for FP32
// vectors, a float-pair split; both run on GB300's narrow FP64/conversion
// path, so doing them once per block instead of once per thread removes a
// fixed cost of several microseconds per launch.  Call from block-uniform
// control flow (it synchronises the block), at most once per call site.
template <typename V, typename F>
__device__ __forceinline__ V block_bcast(F f) {
  __shared__ __align__(16) unsigned char buf[sizeof(V)];
  if (threadIdx.x == 0) {
    const V v = f();
    memcpy(buf, &v, sizeof(V));
  }
  __syncthreads();
  V out = *reinterpret_cast<const V*>(buf);
  return out;
}

// 16-byte vectors of T for the streaming solver kernels: VN elements per
// load/store (2 doubles or 4 floats).  The vector path runs when every
// pointer of the kernel is 16-byte aligned; the last n % VN elements and
// unaligned callers take the scalar path.
template <typename T>
struct Vec16 {
  static constexpr int N = 16 / sizeof(T);
  T v[16 / sizeof(T)];
};
template <typename T>
__device__ __forceinline__ Vec16<T> vload(const T* p) {
  Vec16<T> r;
  if constexpr (sizeof(T) == 8) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    r.v[0] = t.x;
    r.v[1] = t.y;
  } else {
    const float4 t = *reinterpret_cast<const float4*>(p);
    r.v[0] = t.x;
    r.v[1] = t.y;
    r.v[2] = t.z;
    r.v[3] = t.w;
  }
  return r;
}
template <typename T>
__device__ __forceinline__ void vstore(T* p, const Vec16<T>& r) {
  if constexpr (sizeof(T) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(r.v[0], r.v[1]);
  } else {
    *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  }
}
__device__ __forceinline__ bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// vf(i0) handles elements i0 .. i0+VN-1 (16-byte aligned); sf(i) one element.
template <typename T, typename VF, typename SF>
__device__ __forceinline__ void vec_loop(int64_t n, bool aligned, VF vf, SF sf) {
  constexpr int VN = Vec16<T>::N;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  int64_t done = 0;
  if (aligned) {
    const int64_t nv = n / VN;
    int64_t iv = tid;
    // four vectors per trip keep several 16-byte loads in flight per thread
    for (; iv + 3 * nth < nv; iv += 4 * nth) {
      vf(iv * VN);
      vf((iv + nth) * VN);
      vf((iv + 2 * nth) * VN);
      vf((iv + 3 * nth) * VN);
    }
    for (; iv < nv; iv += nth) vf(iv * VN);
    done = nv * VN;
  }
  for (int64_t i = done + tid; i < n; i += nth) sf(i);
}

template <int NV, typename Op>
__device__ __forceinline__ void reduce_op(double (&v)[NV], RedWs ws, Op op) {
  grid_reduce<256, NV>(v, ws.partials, ws.counter, blockIdx.x, gridDim.x, op);
}

#define GKO_GRID_LOOP(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// --------------------------------------------------------------- shared --

// r = b - q (q = A x0, or zero when q == nullptr); copies of r into c1/c2
// (optional), zeroes z1/z2 (optional).  Reduces ||b||^2, ||r||^2.
struct InitOp {
  Ctl* c;
  double rel_tol;
  int kind;  // 0 CG, 1 BiCGSTAB, 2 GMRES (GMRES runs its own restart step)
  // t[0] = b.b, t[1] = r.r, t[2] = r.z (z = M^-1 r with a preconditioner, else r)
  __device__ void operator()(const double (&t)[3]) const {
    c->nb = sqrt(t[0]);
    c->tol_abs = rel_tol * c->nb;
    c->rr = t[1];
    c->iter = 0;
    c->cycles = 0;
    c->phase = 0;
    c->replace = 0;
    if (t[0] == 0.0) {  // b == 0: x = 0 after 0 iterations
      c->status = kConverged;
      c->done = 1;
      return;
    }
    if (sqrt(t[1]) <= c->tol_abs) {
      c->status = kConverged;
      c->done = 1;
      return;
    }
    c->status = kRun;
    c->done = 0;
    c->maxrr = sqrt(t[1]);
    c->half = 0;
    if (kind == 0) {
      c->rho = t[2];
    } else if (kind == 1) {
      c->rho = c->alpha = c->omega = 1.0;
      c->rho_new = t[1];  // rhat = r
      c->beta = t[1];
    }
  }
};

// c1 receives z = d * r when the Jacobi inverse diagonal d is given (CG's
// first direction), else a copy of r.
template <typename T>
__global__ void __launch_bounds__(256, 4) init_residual_kernel(int64_t n, const double* __restrict__ b,
                                                            const T* __restrict__ q, T* __restrict__ r, T* c1, T* c2,
                                                            T* z1, T* z2, RedWs ws, InitOp op,
                                                            const T* __restrict__ d = nullptr) {
  double acc[3] = {0.0, 0.0, 0.0};
  GKO_GRID_LOOP(i, n) {
    const double bi = b[i];
    const T ri = (T)(q ? bi - wd(q[i]) : bi);
    const T zi = d ? d[i] * ri : ri;
    r[i] = ri;
    if (c1) c1[i] = zi;
    if (c2) c2[i] = ri;
    if (z1) z1[i] = T(0);
    if (z2) z2[i] = T(0);
    acc[0] += bi * bi;
    acc[1] += wd(ri) * wd(ri);
    acc[2] += wd(ri) * wd(zi);
  }
  reduce_op<3>(acc, ws, op);
}

// t = b - q stored into q; ||t||^2 decides: converged, or replace r by t.
// t[0] = ||t||^2, t[1] = t.(d t) (= t[0] without a preconditioner)
struct TrueResOp {
  Ctl* c;
  __device__ void operator()(const double (&t)[2]) const {
    if (sqrt(t[0]) <= c->tol_abs) {
      c->status = kConverged;
      c->done = 1;
    } else {
      c->status = kRun;
      c->done = 0;
      c->replace = 1;
      c->rho_new = t[1];
      c->phase = 0;
    }
  }
};

template <typename T>
__global__ void __launch_bounds__(256, 4) true_res_kernel(int64_t n, const double* __restrict__ b, T* __restrict__ q,
                                                       RedWs ws, TrueResOp op, const T* __restrict__ d = nullptr) {
  double acc[2] = {0.0, 0.0};
  GKO_GRID_LOOP(i, n) {
    const T t = (T)(b[i] - wd(q[i]));
    q[i] = t;
    acc[0] += wd(t) * wd(t);
    acc[1] += wd(t) * wd(d ? d[i] * t : t);
  }
  reduce_op<2>(acc, ws, op);
}

// red[0] = w.y, red[1] = y.y (formats whose SpMV cannot fuse the dot).
struct Store2 {
  double* out;
  __device__ void operator()(const double (&t)[2]) const {
    out[0] = t[0];
    out[1] = t[1];
  }
};

template <typename T>
__global__ void __launch_bounds__(256, 4) dot2_kernel(int64_t n, const T* __restrict__ w, const T* __restrict__ y,
                                                   RedWs ws, double* out, const int* gate) {
  pdl_begin();
  if (gated(gate)) return;
  double acc[2] = {0.0, 0.0};
  GKO_GRID_LOOP(i, n) {
    const double yi = wd(y[i]);
    acc[0] += wd(w[i]) * yi;
    acc[1] += yi * yi;
  }
  reduce_op<2>(acc, ws, Store2{out});
}

// ------------------------------------------------------- block-Jacobi --

// z = M^-1 v for block-Jacobi (M = the diagonal blocks of A, Saad Sec.
// 12.2): z_i = sum_j B[i*bs + j] v[base + j] over the nb rows of i's block
// (base = i - i % bs), accumulated in T (FP64 solves: the inverse blocks of
// block_jacobi_inverse; FP32 recurrences: their FP32 rounding, FP32 FMAs).  z2 (nullable) also receives z.  With a reducing
// Op, v.z is reduced into it.  gate: skip while its words are set (the
// iteration kernels); need (nullable): skip unless *need is set (the
// residual replacement after a true-residual check).  Op = NoOp: no
// reduction.

// CG start: rho = r.z
struct BjInitOp {
  Ctl* c;
  __device__ void operator()(const double (&t)[1]) const { c->rho = t[0]; }
};

// CG step: beta = (r.z)_new / (r.z)_old (Saad Alg. 9.1)
struct BjStepOp {
  Ctl* c;
  __device__ void operator()(const double (&t)[1]) const {
    const double rho_new = t[0];
    c->rho_new = rho_new;
    c->beta = rho_new / c->rho;
    c->rho = rho_new;
  }
};

// CG residual replacement: the replaced residual's t.z
struct BjReplaceOp {
  Ctl* c;
  __device__ void operator()(const double (&t)[1]) const { c->rho_new = t[0]; }
};

// BS > 0: the block size as a compile-time constant (rows of full blocks
// then issue all their loads before the first FMA, and each thread takes
// two rows per trip); BS = 0: any block size.
template <typename T, typename Op, int BS = 0>
__global__ void __launch_bounds__(256, 4) bj_apply_kernel(int64_t n, int bs, const T* __restrict__ B,
                                                       const T* __restrict__ v, T* __restrict__ z,
                                                       T* __restrict__ z2, RedWs ws, Op op, const int* gate,
                                                       const int* need) {
  constexpr bool RED = !std::is_same<Op, NoOp>::value;
  pdl_begin();
  if (gated(gate)) return;
  if (need && !*(volatile const int*)need) return;
  constexpr int VN = Vec16<T>::N;
  if (BS) bs = BS;
  // Blocks of a power-of-two size start at i & -bs; blocks whose size is a
  // multiple of VN read their B row and the block of v with 16-byte loads
  // (the row and the block start 16-byte aligned: B and v are 256-byte
  // aligned allocations), the same FMAs in the same order.
  const bool pow2 = (bs & (bs - 1)) == 0;
  const bool vec = bs % VN == 0 && al16(B) && al16(v);
  double acc[1] = {0.0};
  auto row_sum = [&](int64_t i) -> T {
    const int64_t base = pow2 ? (i & ~(int64_t)(bs - 1)) : (int64_t)((int32_t)i / bs) * bs;
    const int nb = (int)(n - base < bs ? n - base : bs);
    const T* Bi = B + i * bs;
    T sum = T(0);
    if (vec && nb == bs) {
      if constexpr (BS > 0 && BS % VN == 0) {
        Vec16<T> bv[BS / VN], xv[BS / VN];
#pragma unroll
        for (int j = 0; j < BS / VN; ++j) {
          bv[j] = vload(Bi + j * VN);
          xv[j] = vload(v + base + j * VN);
        }
#pragma unroll
        for (int j = 0; j < BS / VN; ++j)
#pragma unroll
          for (int k = 0; k < VN; ++k) sum = madd(bv[j].v[k], xv[j].v[k], sum);
      } else {
        for (int j = 0; j < bs; j += VN) {
          const Vec16<T> bv = vload(Bi + j), xv = vload(v + base + j);
#pragma unroll
          for (int k = 0; k < VN; ++k) sum = madd(bv.v[k], xv.v[k], sum);
        }
      }
    } else {
      for (int j = 0; j < nb; ++j) sum = madd(Bi[j], v[base + j], sum);
    }
    return sum;
  };
  auto finish = [&](int64_t i, T zi) {
    z[i] = zi;
    if (z2) z2[i] = zi;
    if (RED) acc[0] = __fma_rn(wd(v[i]), wd(zi), acc[0]);
  };
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if constexpr (BS > 0) {
    for (; i + nth < n; i += 2 * nth) {  // rows in the same order as the loop below
      const T z0 = row_sum(i), z1 = row_sum(i + nth);
      finish(i, z0);
      finish(i + nth, z1);
    }
  }
  for (; i < n; i += nth) finish(i, row_sum(i));
  if constexpr (RED) reduce_op<1>(acc, ws, op);
}

// Launch of bj_apply_kernel with the block size as a template argument
// where it is a common one (FP64 up to 8, FP32 up to 16: the row's B and v
// values stay in registers), else the general kernel.
template <typename T, typename Op>
static cudaError_t bj_launch(dim3 grid, cudaStream_t s, int64_t n, int bs, const T* B, const T* v, T* z, T* z2,
                             RedWs ws, Op op, const int* gate, const int* need) {
  const dim3 blk(256);
  switch (bs) {
    case 4:
      return launch_k(bj_apply_kernel<T, Op, 4>, grid, blk, 0, s, n, bs, B, v, z, z2, ws, op, gate, need);
    case 8:
      return launch_k(bj_apply_kernel<T, Op, 8>, grid, blk, 0, s, n, bs, B, v, z, z2, ws, op, gate, need);
    case 16:
      if constexpr (sizeof(T) == 4)
        return launch_k(bj_apply_kernel<T, Op, 16>, grid, blk, 0, s, n, bs, B, v, z, z2, ws, op, gate, need);
      break;
    default:
      break;
  }
  return launch_k(bj_apply_kernel<T, Op, 0>, grid, blk, 0, s, n, bs, B, v, z, z2, ws, op, gate, need);
}

// Reliable-update test after a step with recurrence residual norm nr (mixed
// precision only; delta = 0 disables it): nr raises maxrr, and nr below
// delta * maxrr asks the host for an update (kCheck, as at convergence).
__device__ __forceinline__ bool reliable_due(Ctl* c, double nr) {
  if (!(c->delta > 0.0)) return false;
  if (nr > c->maxrr) c->maxrr = nr;
  if (nr < c->delta * c->maxrr) {
    c->status = kCheck;
    c->done = 1;
    return true;
  }
  return false;
}

// ------------------------------------------------------------------- CG --

// t[0] = r.r (convergence); with a preconditioner t[1] = r.z (the new rho).
// LATER (block-Jacobi): beta and rho come from the following block-Jacobi
// kernel, which forms z = M^-1 r and r.z.
template <int NV, bool LATER = false>
struct CgUpdateOp {
  Ctl* c;
  __device__ void operator()(const double (&t)[NV]) const {
    const double pq = c->red[0];
    if (!(pq > 0.0)) {
      c->status = kBreakdown;
      c->done = 1;
      return;
    }
    const double rho_new = t[NV - 1];
    c->iter += 1;
    c->rho_new = rho_new;
    const double nr = sqrt(t[0]);
    if (nr <= c->tol_abs) {
      c->status = c->check_true ? kCheck : kConverged;
      c->done = 1;
      return;
    }
    if (reliable_due(c, nr)) return;
    if (c->iter >= c->maxit) {
      c->status = kNotConverged;
      c->done = 1;
      return;
    }
    if (LATER) return;
    c->beta = rho_new / c->rho;
    c->rho = rho_new;
  }
};

// alpha = rho / (p.q); x += alpha p; r -= alpha q; reduces r.r and, with
// the Jacobi inverse diagonal d (PC), r.z for z = d r.  BJ: r.r only, the
// step scalars left to the block-Jacobi kernel that follows.
template <typename T, bool PC, bool BJ = false>
__global__ void __launch_bounds__(256, 4) cg_update_kernel(int64_t n, T* __restrict__ x, T* __restrict__ r,
                                                        const T* __restrict__ p, const T* __restrict__ q, Ctl* c,
                                                        RedWs ws, const T* __restrict__ d) {
  pdl_begin();
  constexpr int NV = PC ? 2 : 1;
  if (gated(&c->done)) return;
  const bool ok = c->red[0] > 0.0;
  const LinPair<T> L = block_bcast<LinPair<T>>([&] {
    const double alpha = ok ? c->rho / c->red[0] : 0.0;
    return LinPair<T>{Lin<T>(alpha), Lin<T>(-alpha)};
  });
  double acc[NV] = {};
  if (ok) {
    const Lin<T> ax = L.a, ar = L.b;
    const bool aligned = al16(x) && al16(r) && al16(p) && al16(q) && (!PC || al16(d));
    vec_loop<T>(n, aligned, [&](int64_t i0) {
          Vec16<T> xv = vload(x + i0), rv = vload(r + i0), dv;
          const Vec16<T> pv = vload(p + i0), qv = vload(q + i0);
          if (PC) dv = vload(d + i0);
#pragma unroll
          for (int k = 0; k < Vec16<T>::N; ++k) {
            xv.v[k] = ax(pv.v[k], xv.v[k]);
            rv.v[k] = ar(qv.v[k], rv.v[k]);
            const double rw = wd(rv.v[k]);
            acc[0] = __fma_rn(rw, rw, acc[0]);
            if (PC) acc[NV - 1] = __fma_rn(rw, wd(dv.v[k] * rv.v[k]), acc[NV - 1]);
          }
          vstore(x + i0, xv);
          vstore(r + i0, rv);
        }, [&](int64_t i) {
          x[i] = ax(p[i], x[i]);
          const T ri = ar(q[i], r[i]);
          r[i] = ri;
          const double rw = wd(ri);
          acc[0] = __fma_rn(rw, rw, acc[0]);
          if (PC) acc[NV - 1] = __fma_rn(rw, wd(d[i] * ri), acc[NV - 1]);
        });
  }
  reduce_op<NV>(acc, ws, CgUpdateOp<NV, BJ>{c});
}

// p = z + beta p, z = d r with the Jacobi inverse diagonal (PC), else r
template <typename T, bool PC>
__global__ void __launch_bounds__(256, 4) cg_p_kernel(int64_t n, const T* __restrict__ r, T* __restrict__ p, Ctl* c,
                                                   const T* __restrict__ d) {
  pdl_begin();
  if (gated(&c->done)) return;
  const Lin<T> bp = block_bcast<Lin<T>>([&] { return Lin<T>(c->beta); });
  const bool aligned = al16(r) && al16(p) && (!PC || al16(d));
  vec_loop<T>(n, aligned, [&](int64_t i0) {
        Vec16<T> pv = vload(p + i0);
        const Vec16<T> rv = vload(r + i0);
        Vec16<T> dv;
        if (PC) dv = vload(d + i0);
#pragma unroll
        for (int k = 0; k < Vec16<T>::N; ++k) pv.v[k] = bp(pv.v[k], PC ? dv.v[k] * rv.v[k] : rv.v[k]);
        vstore(p + i0, pv);
      }, [&](int64_t i) { p[i] = bp(p[i], PC ? d[i] * r[i] : r[i]); });
}

// after a failed true-residual check: r = t, beta = rho_new/rho, p = r + beta p
struct CgReplaceOp {
  Ctl* c;
  __device__ void operator()(const double (&)[1]) const {
    c->replace = 0;
    c->rho = c->rho_new;
  }
};

// z (block-Jacobi, nullable): the preconditioned t, p = z + beta p
template <typename T>
__global__ void __launch_bounds__(256, 4) cg_replace_kernel(int64_t n, T* __restrict__ r, T* __restrict__ p,
                                                         const T* __restrict__ t, Ctl* c, RedWs ws,
                                                         const T* __restrict__ d = nullptr,
                                                         const T* __restrict__ z = nullptr) {
  if (!*(volatile int*)&c->replace) return;
  const Lin<T> bp = block_bcast<Lin<T>>([&] { return Lin<T>(c->rho_new / c->rho); });
  double acc[1] = {0.0};
  GKO_GRID_LOOP(i, n) {
    const T ri = t[i];
    r[i] = ri;
    p[i] = bp(p[i], z ? z[i] : (d ? d[i] * ri : ri));
  }
  reduce_op<1>(acc, ws, CgReplaceOp{c});
}

// ------------------------------------------------------------- BiCGSTAB --

// p = r + beta (p - omega v); with the Jacobi inverse diagonal d also the
// preconditioned direction ph = d p (right preconditioning)
template <typename T>
__global__ void __launch_bounds__(256, 4) bicg_p_kernel(int64_t n, const T* __restrict__ r, T* __restrict__ p,
                                                     const T* __restrict__ v, Ctl* c, const T* __restrict__ d = nullptr,
                                                     T* __restrict__ ph = nullptr) {
  pdl_begin();
  if (gated(&c->done)) return;
  const LinPair<T> L = block_bcast<LinPair<T>>([&] { return LinPair<T>{Lin<T>(c->beta), Lin<T>(-c->omega)}; });
  const Lin<T> bp = L.a, wv = L.b;
  if (d) {
    GKO_GRID_LOOP(i, n) {
      const T pi = bp(wv(v[i], p[i]), r[i]);
      p[i] = pi;
      ph[i] = d[i] * pi;
    }
    return;
  }
  const bool aligned = al16(r) && al16(p) && al16(v);
  vec_loop<T>(n, aligned, [&](int64_t i0) {
        Vec16<T> pv = vload(p + i0);
        const Vec16<T> rv = vload(r + i0), vv = vload(v + i0);
#pragma unroll
        for (int k = 0; k < Vec16<T>::N; ++k) pv.v[k] = bp(wv(vv.v[k], pv.v[k]), rv.v[k]);
        vstore(p + i0, pv);
      }, [&](int64_t i) { p[i] = bp(wv(v[i], p[i]), r[i]); });
}

struct BicgSOp {
  Ctl* c;
  __device__ void operator()(const double (&t)[1]) const {
    const double rv = c->red[0];
    if (rv == 0.0) {
      c->status = kBreakdown;
      c->done = 1;
      return;
    }
    c->alpha = c->rho_new / rv;
    c->iter += 1;
    if (sqrt(t[0]) <= c->tol_abs) c->phase = 1;  // finish with x += alpha p
  }
};

// alpha = rho_new / (rhat.v); s = r - alpha v; reduces s.s
template <typename T>
__global__ void __launch_bounds__(256, 4) bicg_s_kernel(int64_t n, const T* __restrict__ r, const T* __restrict__ v,
                                                     T* __restrict__ s, Ctl* c, RedWs ws,
                                                     const T* __restrict__ d = nullptr, T* __restrict__ sh = nullptr) {
  pdl_begin();
  if (gated(&c->done)) return;
  const double rv = c->red[0];
  const Lin<T> av = block_bcast<Lin<T>>([&] { return Lin<T>(rv != 0.0 ? -(c->rho_new / rv) : 0.0); });
  double acc[1] = {0.0};
  if (rv != 0.0 && d) {  // right preconditioning: also sh = d s
    GKO_GRID_LOOP(i, n) {
      const T si = av(v[i], r[i]);
      s[i] = si;
      sh[i] = d[i] * si;
      const double sw = wd(si);
      acc[0] = __fma_rn(sw, sw, acc[0]);
    }
  } else if (rv != 0.0) {
    const bool aligned = al16(r) && al16(v) && al16(s);
    vec_loop<T>(n, aligned, [&](int64_t i0) {
          const Vec16<T> vv = vload(v + i0), rr = vload(r + i0);
          Vec16<T> sv;
#pragma unroll
          for (int k = 0; k < Vec16<T>::N; ++k) {
            sv.v[k] = av(vv.v[k], rr.v[k]);
            const double sw = wd(sv.v[k]);
            acc[0] = __fma_rn(sw, sw, acc[0]);
          }
          vstore(s + i0, sv);
        }, [&](int64_t i) {
          const T si = av(v[i], r[i]);
          s[i] = si;
          const double sw = wd(si);
          acc[0] = __fma_rn(sw, sw, acc[0]);
        });
  }
  reduce_op<1>(acc, ws, BicgSOp{c});
}

struct BicgXOp {
  Ctl* c;
  __device__ void operator()(const double (&t)[2]) const {
    if (c->phase) {  // half step: ||s|| small, x += alpha p was done
      c->phase = 0;
      c->half = 1;
      c->status = c->check_true ? kCheck : kConverged;
      c->done = 1;
      return;
    }
    c->half = 0;
    const double tt = c->red[1];
    if (tt == 0.0) {
      c->status = kBreakdown;
      c->done = 1;
      return;
    }
    const double omega = c->red[0] / tt;
    c->omega = omega;
    c->rho = c->rho_new;
    c->rho_new = t[1];
    const double nr = sqrt(t[0]);
    if (nr <= c->tol_abs) {
      c->status = c->check_true ? kCheck : kConverged;
      c->done = 1;
      return;
    }
    if (reliable_due(c, nr)) return;
    if (omega == 0.0 || (c->iter < c->maxit && c->rho_new == 0.0)) {
      c->status = kBreakdown;
      c->done = 1;
      return;
    }
    if (c->iter >= c->maxit) {
      c->status = kNotConverged;
      c->done = 1;
      return;
    }
    c->beta = (c->rho_new / c->rho) * (c->alpha / omega);
  }
};

// omega = t.s / t.t; x += alpha p + omega s; r = s - omega t; reduces r.r and
// rhat.r.  In the half step only x += alpha p.  Right preconditioning: x
// moves along ph = d p and sh = d s instead.
template <typename T>
__global__ void __launch_bounds__(256, 4) bicg_x_kernel(int64_t n, T* __restrict__ x, const T* __restrict__ p,
                                                     const T* __restrict__ s, const T* __restrict__ t,
                                                     T* __restrict__ r, const T* __restrict__ rh, Ctl* c, RedWs ws,
                                                     const T* __restrict__ ph = nullptr,
                                                     const T* __restrict__ sh = nullptr) {
  pdl_begin();
  if (gated(&c->done)) return;
  double acc[2] = {0.0, 0.0};
  const LinTriple<T> L = block_bcast<LinTriple<T>>([&] {
    const double tt = c->red[1];
    const double omega = tt != 0.0 ? c->red[0] / tt : 0.0;
    return LinTriple<T>{Lin<T>(c->alpha), Lin<T>(omega), Lin<T>(-omega)};
  });
  const Lin<T> ap = L.a;
  if (*(volatile int*)&c->phase) {
    const T* xp = ph ? ph : p;
    GKO_GRID_LOOP(i, n) x[i] = ap(xp[i], x[i]);
  } else if (ph) {
    const double tt = c->red[1];
    if (tt != 0.0) {
      const Lin<T> os = L.b, ot = L.c;
      GKO_GRID_LOOP(i, n) {
        x[i] = os(sh[i], ap(ph[i], x[i]));
        const T ri = ot(t[i], s[i]);
        r[i] = ri;
        const double rw = wd(ri);
        acc[0] = __fma_rn(rw, rw, acc[0]);
        acc[1] = __fma_rn(wd(rh[i]), rw, acc[1]);
      }
    }
  } else {
    const double tt = c->red[1];
    if (tt != 0.0) {
      const Lin<T> os = L.b, ot = L.c;
      const bool aligned = al16(x) && al16(p) && al16(s) && al16(t) && al16(r) && al16(rh);
      vec_loop<T>(n, aligned, [&](int64_t i0) {
            Vec16<T> xv = vload(x + i0), rv;
            const Vec16<T> sv = vload(s + i0), pv = vload(p + i0), tv = vload(t + i0), hv = vload(rh + i0);
#pragma unroll
            for (int k = 0; k < Vec16<T>::N; ++k) {
              xv.v[k] = os(sv.v[k], ap(pv.v[k], xv.v[k]));
              rv.v[k] = ot(tv.v[k], sv.v[k]);
              const double rw = wd(rv.v[k]);
              acc[0] = __fma_rn(rw, rw, acc[0]);
              acc[1] = __fma_rn(wd(hv.v[k]), rw, acc[1]);
            }
            vstore(x + i0, xv);
            vstore(r + i0, rv);
          }, [&](int64_t i) {
            const T si = s[i];
            x[i] = os(si, ap(p[i], x[i]));
            const T ri = ot(t[i], si);
            r[i] = ri;
            const double rw = wd(ri);
            acc[0] = __fma_rn(rw, rw, acc[0]);
            acc[1] = __fma_rn(wd(rh[i]), rw, acc[1]);
          });
    }
  }
  reduce_op<2>(acc, ws, BicgXOp{c});
}

// after a failed true-residual check: restart the recurrences from r = t
struct BicgRestartOp {
  Ctl* c;
  __device__ void operator()(const double (&t)[1]) const {
    c->replace = 0;
    c->rho = c->alpha = c->omega = 1.0;
    c->rho_new = t[0];
    c->beta = t[0];
    if (c->iter >= c->maxit) {
      c->status = kNotConverged;
      c->done = 1;
    } else if (t[0] == 0.0) {
      c->status = kBreakdown;
      c->done = 1;
    }
  }
};

template <typename T>
__global__ void __launch_bounds__(256, 4) bicg_restart_kernel(int64_t n, T* __restrict__ r, const T* __restrict__ rh,
                                                           T* __restrict__ p, T* __restrict__ v,
                                                           const T* __restrict__ t, Ctl* c, RedWs ws) {
  if (!*(volatile int*)&c->replace) return;
  double acc[1] = {0.0};
  GKO_GRID_LOOP(i, n) {
    const T ri = t[i];
    r[i] = ri;
    p[i] = T(0);
    v[i] = T(0);
    acc[0] += wd(rh[i]) * wd(ri);
  }
  reduce_op<1>(acc, ws, BicgRestartOp{c});
}

// ------------------------------------------------------ reliable updates --
//
// Mixed-precision CG / BiCGSTAB with reliable updates (Sleijpen & van der
// Vorst 1996; residual replacement without restart as in van der Vorst & Ye
// 2000): the recurrences run on the FP32 copy of A with FP32 vectors and
// accumulate the iterate's change d; an update folds d into the FP64
// solution and replaces the recurrence residual by the FP64 residual
// b - A x, keeping the directions and scalars (BiCGSTAB restarts only after
// its half step, whose s has no continuation).

// x64 += d (exact widening), d = 0
__global__ void __launch_bounds__(256, 4) fold_kernel(int64_t n, double* __restrict__ x64, float* __restrict__ d) {
  GKO_GRID_LOOP(i, n) {
    x64[i] += widen(d[i]);
    d[i] = 0.0f;
  }
}

// t[0] = ||b - A x||^2 (FP64), t[1] = rhat.r (BiCGSTAB) or r.z (CG) of the
// replaced, rounded residual r.
struct RelOp {
  Ctl* c;
  int solver;
  int half;
  __device__ void operator()(const double (&t)[2]) const {
    const double rn = sqrt(t[0]);
    c->phase = 0;
    c->half = 0;
    if (rn <= c->tol_abs) {
      c->status = kConverged;
      c->done = 1;
      return;
    }
    c->maxrr = rn;
    c->status = kRun;
    c->done = 0;
    if (solver == 0) {  // CG: cg_replace_kernel finishes (r = t, p = z + beta p)
      if (c->iter >= c->maxit) {
        c->status = kNotConverged;
        c->done = 1;
        return;
      }
      c->replace = 1;
      c->rho_new = t[1];
      return;
    }
    if (half) {  // BiCGSTAB after a half step: bicg_restart_kernel restarts
      c->replace = 1;
      return;
    }
    if (c->omega == 0.0) {
      c->status = kBreakdown;
      c->done = 1;
      return;
    }
    if (c->iter >= c->maxit) {
      c->status = kNotConverged;
      c->done = 1;
      return;
    }
    c->rho_new = t[1];
    if (t[1] == 0.0) {
      c->status = kBreakdown;
      c->done = 1;
      return;
    }
    c->beta = (c->rho_new / c->rho) * (c->alpha / c->omega);
  }
};

// dst = fl(b - q) with q = A64 x64; reduces ||b - q||^2 in FP64 and
// w.dst (w = rhat for BiCGSTAB) or dst.(d dst) (CG, d the Jacobi diagonal
// or none).
template <typename T>
__global__ void __launch_bounds__(256, 4) rel_replace_kernel(int64_t n, const double* __restrict__ b,
                                                          const double* __restrict__ q, T* __restrict__ dst,
                                                          const T* __restrict__ w, const T* __restrict__ d,
                                                          RedWs ws, RelOp op) {
  double acc[2] = {0.0, 0.0};
  GKO_GRID_LOOP(i, n) {
    const double ti = b[i] - q[i];
    const T tr = (T)ti;
    dst[i] = tr;
    acc[0] = __fma_rn(ti, ti, acc[0]);
    const double tw = wd(tr);
    acc[1] = __fma_rn(w ? wd(w[i]) : tw, w ? tw : wd(d ? d[i] * tr : tr), acc[1]);
  }
  reduce_op<2>(acc, ws, op);
}

// What a reliable-update solve needs beyond the recurrences' operator.
struct RelSpec {
  const gko_matrix_s* A64;  // FP64 matrix for the replaced residuals
  const double* b64;        // right-hand side
  double* x64;              // FP64 solution (x0 on entry)
  double* q64;              // n doubles of workspace
  void* scratch;            // SpMV scratch of A64
  double delta;
};

// ---------------------------------------------------------------- GMRES --

// Cycle start: v0 = r = b - A x (q = A x), ||r|| -> beta, g = beta e1.
struct GmStartOp {
  Ctl* c;
  double* g;
  int m;
  __device__ void operator()(const double (&t)[1]) const {
    const double beta = sqrt(t[0]);
    c->rr = t[0];
    c->phase = 0;
    c->k = 0;
    if (beta <= c->tol_abs) {
      c->status = kConverged;
      c->done = 1;
      return;
    }
    if (c->iter >= c->maxit) {
      c->status = kNotConverged;
      c->done = 1;
      return;
    }
    c->beta = beta;
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
  }
};

template <typename T>
__global__ void __launch_bounds__(256, 4) gm_start_kernel(int64_t n, const double* __restrict__ b,
                                                       const T* __restrict__ q, T* __restrict__ v0, Ctl* c, RedWs ws,
                                                       GmStartOp op) {
  if (gated(&c->done)) return;
  double acc[1] = {0.0};
  GKO_GRID_LOOP(i, n) {
    const T ri = (T)(q ? b[i] - wd(q[i]) : b[i]);
    v0[i] = ri;
    acc[0] += wd(ri) * wd(ri);
  }
  reduce_op<1>(acc, ws, op);
}

// v = v * (1 / *den); den = &beta for v0, &H[(j+1), j] for v_{j+1}
template <typename T>
__global__ void __launch_bounds__(256, 4) gm_scale_kernel(int64_t n, T* __restrict__ v, const double* den, Ctl* c) {
  if (gated(&c->phase)) return;
  const Lin<T> sc = block_bcast<Lin<T>>([&] { return Lin<T>(1.0 / *den); });
  GKO_GRID_LOOP(i, n) v[i] = sc.scale(v[i]);
}

// gated multi-dot: partial sums of V_j . w for j <= jmax (blockIdx.y = j)
template <typename T>
__global__ void __launch_bounds__(256, 4) gm_multidot_kernel(int64_t n, const T* __restrict__ V, int64_t ldv,
                                                          const T* __restrict__ w, double* __restrict__ partials,
                                                          Ctl* c, int pass) {
  pdl_begin();
  if (gated(&c->phase) || (pass == 1 && *(volatile int*)&c->noreorth)) return;
  const int j = blockIdx.y;
  const T* v = V + (int64_t)j * ldv;
  double acc = 0.0;
  GKO_GRID_LOOP(i, n) acc = __fma_rn(wd(v[i]), wd(__ldg(w + i)), acc);
  const double sblk = block_sum<256>(acc);
  if (threadIdx.x == 0) partials[(int64_t)j * kMultiSlots + blockIdx.x] = sblk;
}

__global__ void __launch_bounds__(256, 4) gm_multidot_finish_kernel(int g, const double* __restrict__ partials,
                                                                 double* __restrict__ h, int accumulate, Ctl* c,
                                                                 int pass) {
  pdl_begin();
  if (gated(&c->phase) || (pass == 1 && *(volatile int*)&c->noreorth)) return;
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < g; i += 256) acc += partials[(int64_t)j * kMultiSlots + i];
  const double t = block_sum<256>(acc);
  if (threadIdx.x == 0) h[j] = accumulate ? h[j] + t : t;
}

struct StoreRr {
  Ctl* c;
  int decide;  // first pass: skip the second pass unless ||w|| fell below ||w0|| / sqrt(2)
  __device__ void operator()(const double (&t)[1]) const {
    c->rr = t[0];
    if (decide) c->noreorth = t[0] >= 0.5 * c->red[0] ? 1 : 0;
  }
};

// w -= sum_{j<=jmax} h_j V_j (h: device, the pass's coefficients); with
// NORM also reduces ||w||^2 into c->rr.
constexpr int kMaxRestart = 128;

// -h_j as the coefficient pair of Lin<T>, built once per block
template <typename T>
__device__ __forceinline__ void load_coefs(const double* h, int count, double sign, T* hi, T* lo) {
  for (int j = threadIdx.x; j < count; j += blockDim.x) {
    const double a = sign * h[j];
    if constexpr (sizeof(T) == 4) {
      const float f = __double2float_rn(a);
      hi[j] = f;
      lo[j] = __double2float_rn(a - (double)f);
    } else {
      hi[j] = a;
      lo[j] = 0.0;
    }
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ T lin_apply(T hi, T lo, T x, T y) {
  if constexpr (sizeof(T) == 4) return __fmaf_rn(lo, x, __fmaf_rn(hi, x, y));
  else return __fma_rn(hi, x, y);
}

template <typename T, bool NORM>
__global__ void __launch_bounds__(256, 4) gm_axpy_kernel(int64_t n, int jcount, const double* __restrict__ h,
                                                      const T* __restrict__ V, int64_t ldv, T* __restrict__ w, Ctl* c,
                                                      RedWs ws, int pass) {
  pdl_begin();
  __shared__ T s_hi[kMaxRestart + 1], s_lo[kMaxRestart + 1];
  if (gated(&c->phase) || (pass == 1 && *(volatile int*)&c->noreorth)) return;
  load_coefs<T>(h, jcount, -1.0, s_hi, s_lo);
  double acc[1] = {0.0};
  GKO_GRID_LOOP(i, n) {
    T v = w[i];
    for (int j = 0; j < jcount; ++j) v = lin_apply<T>(s_hi[j], s_lo[j], V[(int64_t)j * ldv + i], v);
    w[i] = v;
    if (NORM) {
      const double ow = wd(v);
      acc[0] = __fma_rn(ow, ow, acc[0]);
    }
  }
  if (NORM) reduce_op<1>(acc, ws, StoreRr{c, pass == 0});
}

// Column j of the Hessenberg matrix from the two CGS passes, previous Givens
// rotations, a new rotation, the residual estimate |g_{j+1}| and the cycle
// end test.  One thread.
__global__ void gm_givens_kernel(int j, int m, const double* __restrict__ h1, const double* __restrict__ h2,
                                 double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                                 double* __restrict__ g, Ctl* c) {
  pdl_begin();
  if (gated(&c->phase)) return;
  double* col = H + (int64_t)j;  // H[i*m + j]
  const bool two = !c->noreorth;
  for (int i = 0; i <= j; ++i) col[(int64_t)i * m] = two ? h1[i] + h2[i] : h1[i];
  const double hn = sqrt(c->rr);
  col[(int64_t)(j + 1) * m] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = col[(int64_t)i * m], b = col[(int64_t)(i + 1) * m];
    col[(int64_t)i * m] = cs[i] * a + sn[i] * b;
    col[(int64_t)(i + 1) * m] = -sn[i] * a + cs[i] * b;
  }
  const double a = col[(int64_t)j * m], b = col[(int64_t)(j + 1) * m];
  const double den = sqrt(a * a + b * b);
  c->iter += 1;
  c->k = j + 1;
  if (den == 0.0) {
    c->status = kBreakdown;
    c->k = j;
    c->phase = 1;
    return;
  }
  cs[j] = a / den;
  sn[j] = b / den;
  col[(int64_t)j * m] = den;
  col[(int64_t)(j + 1) * m] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  c->rho = hn;  // h_{j+1,j}, the divisor of the next basis vector
  if (hn == 0.0 || fabs(g[j + 1]) <= c->tol_abs) c->replace = 1;  // estimate says converged
  if (c->replace || c->iter >= c->maxit || j + 1 == m) c->phase = 1;
}

// v_{j+1} = w / h_{j+1,j} (skipped once the cycle has ended)
template <typename T>
__global__ void __launch_bounds__(256, 4) gm_next_kernel(int64_t n, const T* __restrict__ w, T* __restrict__ vn,
                                                      Ctl* c) {
  pdl_begin();
  if (gated(&c->phase)) return;
  const Lin<T> sc = block_bcast<Lin<T>>([&] { return Lin<T>(1.0 / c->rho); });
  GKO_GRID_LOOP(i, n) vn[i] = sc.scale(w[i]);
}

// Back substitution H[0:k,0:k] y = g[0:k]; stores -y for the x update.
__global__ void gm_backsolve_kernel(int m, const double* __restrict__ H, const double* __restrict__ g,
                                    double* __restrict__ ny, Ctl* c) {
  if (gated(&c->done)) return;
  const int k = c->k;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int l = i + 1; l < k; ++l) s -= H[(int64_t)i * m + l] * (-ny[l]);
    ny[i] = -(s / H[(int64_t)i * m + i]);
  }
  c->cycles += 1;
}

// x += V y  (= x - sum_j ny_j V_j), then close the cycle: stop on breakdown,
// otherwise the next cycle recomputes the true residual.
template <typename T>
__global__ void __launch_bounds__(256, 4) gm_update_x_kernel(int64_t n, const double* __restrict__ ny,
                                                          const T* __restrict__ V, int64_t ldv, T* __restrict__ x,
                                                          Ctl* c) {
  __shared__ T s_hi[kMaxRestart + 1], s_lo[kMaxRestart + 1];
  if (gated(&c->done)) return;
  const int k = c->k;
  load_coefs<T>(ny, k, -1.0, s_hi, s_lo);
  GKO_GRID_LOOP(i, n) {
    T v = x[i];
    for (int j = 0; j < k; ++j) v = lin_apply<T>(s_hi[j], s_lo[j], V[(int64_t)j * ldv + i], v);
    x[i] = v;
  }
}

// End of cycle: stop on breakdown; an inner solve (no true-residual check)
// also stops when the Givens estimate met the tolerance.  Otherwise the next
// cycle start recomputes the true residual and decides.
__global__ void gm_close_kernel(Ctl* c) {
  if (gated(&c->done)) return;
  if (c->status == kBreakdown) {
    c->done = 1;
  } else if (!c->check_true && c->replace) {
    c->status = kConverged;
    c->done = 1;
  }
  c->replace = 0;
  c->phase = 0;
}

// ------------------------------------------------------- final residual --

struct FinalOp {
  Ctl* c;
  __device__ void operator()(const double (&t)[1]) const { c->rr = t[0]; }
};

template <typename T>
__global__ void __launch_bounds__(256, 4) final_res_kernel(int64_t n, const double* __restrict__ b,
                                                        const T* __restrict__ q, RedWs ws, Ctl* c) {
  double acc[1] = {0.0};
  GKO_GRID_LOOP(i, n) {
    const double t = b[i] - wd(q[i]);
    acc[0] += t * t;
  }
  reduce_op<1>(acc, ws, FinalOp{c});
}

template <typename T>
__global__ void zero_kernel(int64_t n, T* __restrict__ x) {
  GKO_GRID_LOOP(i, n) x[i] = T(0);
}

// x64 += d (mixed precision refinement update)
__global__ void add_f32_kernel(int64_t n, double* __restrict__ x, const float* __restrict__ d) {
  GKO_GRID_LOOP(i, n) x[i] += (double)d[i];
}

// ================================================================ host ====

static int vec_grid(int64_t n) {
  const int64_t g = std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 4));
  return (int)g;
}

// Pinned host mirror of Ctl for polling.
static Ctl* host_ctl() {
  thread_local Ctl* h = nullptr;
  if (!h) {
    if (cudaMallocHost((void**)&h, sizeof(Ctl)) != cudaSuccess) {
      cudaGetLastError();
      static thread_local Ctl fallback;
      h = &fallback;
    }
  }
  return h;
}

static int read_ctl(const Ctl* d, Ctl* h, cudaStream_t s) {
  GKO_TRY_CUDA(cudaMemcpyAsync(h, d, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  return GKO_OK;
}

// A batch of solver iterations captured once as a CUDA graph and replayed:
// every iteration kernel reads its scalars from the device state and is
// gated on it, so the same graph serves every batch of a solve.  Replaying
// it replaces dozens of host launches per batch by one (small systems are
// launch-bound: about 28 us per CG iteration from the host, whatever n).
// Capture is thread-local (serving workers capture on their own streams);
// if the runtime refuses a capture the solve keeps launching directly.
struct BatchGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t e = nullptr;
  bool refused = false;
  BatchGraph() = default;
  BatchGraph(const BatchGraph&) = delete;
  BatchGraph& operator=(const BatchGraph&) = delete;
  ~BatchGraph() {
    if (e) cudaGraphExecDestroy(e);
    if (g) cudaGraphDestroy(g);
  }
  // enqueue(): puts the batch's kernels on s; returns a GKO status
  template <typename F>
  int capture(cudaStream_t s, F&& enqueue) {
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      refused = true;
      return GKO_OK;
    }
    const int rc = enqueue();
    cudaGraph_t gg = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s, &gg);
    if (rc != GKO_OK) {
      if (gg) cudaGraphDestroy(gg);
      return rc;
    }
    if (ec != cudaSuccess || !gg || cudaGraphInstantiate(&e, gg, 0) != cudaSuccess) {
      cudaGetLastError();
      if (gg) cudaGraphDestroy(gg);
      e = nullptr;
      refused = true;
      return GKO_OK;
    }
    g = gg;
    return GKO_OK;
  }
};
constexpr int kGraphIters = 16;  // iterations per replayed batch

// Bump allocator over one pool allocation.
struct Carve {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) / 256 * 256;
    T* p = reinterpret_cast<T*>(base + off);
    off += sizeof(T) * count + 64;
    return p;
  }
};

struct SolveSpec {
  int solver;  // 0 CG, 1 BiCGSTAB, 2 GMRES
  double rel_tol;
  int maxit;
  int restart;
  int check_true;
  int check_every;
  const void* minv = nullptr;  // Jacobi inverse diagonal (vector of T), or none
  const RelSpec* rel = nullptr;  // reliable updates (FP32 recurrences only)
  const void* bj = nullptr;  // block-Jacobi inverse blocks (n x bs, of T), or none
  int bs = 0;                  // block-Jacobi block size
};

struct SolveOut {
  int status;
  int iterations;
  int cycles;
};

// ------------------------------------------------ single-launch small CG --
//
// Small systems are bound by kernel launch latency, not bandwidth: three
// dependent launches per CG iteration take about 24 us whatever n.  For a
// CSR handle with the row-block plan (regular rows) and n <= kSmallRows, the
// whole CG (Saad Alg. 6.18, Jacobi-preconditioned as Alg. 9.1 when a
// diagonal is given, with the multi-kernel path's true-residual check,
// residual replacement, breakdown and iteration-cap rules) runs in one
// cooperative launch of G blocks.  Thread t of block g owns RPT rows (g *
// 256 * RPT + t + j * 256) and keeps their x, r, p, b and Jacobi entries in
// registers; the block stages its rows' matrix entries in shared memory once
// (when they fit), so an iteration reads only the gathered p values from
// L2.  p is published to global memory after each update, x only for the
// true-residual check and at the end.  Each iteration is the SpMV and two
// grid reductions separated by three grid barriers.  Reductions are
// deterministic: every block adds the G block partials in index order, so
// all blocks hold the same scalars and take the same decisions.  Values
// written by other blocks (the gathered p and x, the partials) are read with
// ld.global.cg: inside one launch L1 is not coherent across SMs.  Every
// barrier wait is bounded (~1 s); a block that gives up records GKO_TIMEOUT
// and the solve returns it.
constexpr int kSmallThreads = 256;
constexpr int64_t kSmallRows = 1 << 18;
constexpr long long kSmallWait = 1ll << 31;
constexpr size_t kSmallSmemMax = 96 * 1024;  // staged matrix entries per block

template <typename T, typename VT>
struct SmallArgs {
  int64_t n;
  const int32_t* rp;
  const int32_t* col;
  const VT* val;
  const double* b;  // FP64 right-hand side
  T* x;
  T* p;
  const T* d;  // Jacobi inverse diagonal, or null
  double rel_tol;
  int maxit;
  int check_true;
  int x_zero;
  int32_t block_cap;  // staged entries per block (shared memory)
  double* part;       // 4 reduction sites x 3 values x gridDim.x
  unsigned* bar;      // grid barrier: arrival counter (zero at launch)
  int* err;
  Ctl* c;             // status and iteration count on exit
};

// Grid-wide barrier of a cooperative launch (all blocks resident), bounded:
// one monotonic arrival counter (zero at launch); barrier number k of the
// launch waits until it reaches (k + 1) * gridDim.x.  Each block's thread 0
// arrives with a release add and polls with acquire loads, so a barrier
// costs about one L2 round trip after the last arrival and nothing is reset.
// `target` is the caller's count of barriers passed times the grid size
// (the same in every thread).
__device__ __forceinline__ bool small_sync(unsigned* bar, unsigned& target, int* err) {
  __shared__ int s_ok;
  target += gridDim.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(bar), "r"(1u) : "memory");
    const long long t0 = clock64();
    for (;;) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if ((int)(v - target) >= 0) break;
      if (clock64() - t0 > kSmallWait) {
        if (err) atomicOr(err, 1 << GKO_TIMEOUT);
        ok = 0;
        break;
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Grid sum of NV values: block sums to part[k * G + block], barrier, then
// every block adds the G partials in index order (warp 0, lane-strided, then
// a fixed butterfly): the same totals in every block.
template <int NV>
__device__ __forceinline__ bool small_reduce(double (&v)[NV], double* part, unsigned* bar, unsigned& target,
                                             int* err) {
  __shared__ double tot[NV];
  block_sum_n<kSmallThreads, NV>(v);
  const int G = gridDim.x;
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) part[(int64_t)k * G + blockIdx.x] = v[k];
  if (!small_sync(bar, target, err)) return false;
  if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int i = threadIdx.x; i < G; i += 32) s += __ldcg(part + (int64_t)k * G + i);
      s = subwarp_sum<32>(s, 0xffffffffu);
      if (threadIdx.x == 0) tot[k] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = tot[k];
  return true;
}

template <typename T, typename VT, int RPT, bool SMEM>
__global__ void __launch_bounds__(kSmallThreads) small_cg_kernel(SmallArgs<T, VT> a) {
  using AT = acc_t<VT>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int G3 = 3 * (int)gridDim.x;
  double* P_init = a.part;
  double* P_pq = a.part + G3;
  double* P_rr = a.part + 2 * G3;
  double* P_true = a.part + 3 * G3;
  const int64_t row0 = (int64_t)blockIdx.x * kSmallThreads * RPT;
  const int64_t row1 = row0 + (int64_t)kSmallThreads * RPT < a.n ? row0 + (int64_t)kSmallThreads * RPT : a.n;
  const int32_t e0 = __ldg(a.rp + row0), e1 = __ldg(a.rp + row1);
  int32_t* scol = reinterpret_cast<int32_t*>(smem_raw);
  VT* sval = reinterpret_cast<VT*>(smem_raw + (((size_t)a.block_cap * sizeof(int32_t) + 15) & ~(size_t)15));
  if (SMEM) {
    for (int32_t k = e0 + (int32_t)threadIdx.x; k < e1; k += kSmallThreads) {
      scol[k - e0] = __ldg(a.col + k);
      sval[k - e0] = a.val[k];
    }
  }
  __syncthreads();
  // this thread's rows
  int32_t ks[RPT], ke[RPT];
  bool own[RPT];
  double bj[RPT];
  T xj[RPT], rj[RPT], pj[RPT], dj[RPT];
#pragma unroll
  for (int j = 0; j < RPT; ++j) {
    const int64_t i = row0 + threadIdx.x + (int64_t)j * kSmallThreads;
    own[j] = i < a.n;
    ks[j] = own[j] ? __ldg(a.rp + i) - (SMEM ? e0 : 0) : 0;
    ke[j] = own[j] ? __ldg(a.rp + i + 1) - (SMEM ? e0 : 0) : 0;
    bj[j] = own[j] ? a.b[i] : 0.0;
    xj[j] = own[j] && !a.x_zero ? a.x[i] : T(0);
    dj[j] = own[j] && a.d ? a.d[i] : T(1);
  }
  const bool pc = a.d != nullptr;
  // row j of A v: staged (or global) entries in storage order, v gathered
  // with ld.global.cg; the gathers of up to 8 entries are issued before
  // their FMAs, so a stencil row costs one L2 round trip, not one per entry
  auto row_dot = [&](int j, const T* v) -> T {
    constexpr int U = 8;
    AT s = AT(0);
    for (int32_t k = ks[j]; k < ke[j]; k += U) {
      VT w[U];
      T g[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool in = k + u < ke[j];
        const int32_t c = in ? (SMEM ? scol[k + u] : __ldg(a.col + k + u)) : 0;
        w[u] = in ? (SMEM ? sval[k + u] : a.val[k + u]) : VT(0);
        g[u] = in ? __ldcg(v + c) : T(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (k + u < ke[j]) s = madd(to_acc(w[u]), to_acc(g[u]), s);
    }
    return (T)s;
  };
  auto publish = [&](T* dst, const T (&v)[RPT]) {
#pragma unroll
    for (int j = 0; j < RPT; ++j)
      if (own[j]) dst[row0 + threadIdx.x + (int64_t)j * kSmallThreads] = v[j];
  };
  int status = kRun, it = 0;
  unsigned tgt = 0;  // grid barriers passed x gridDim.x
  // r = b - A x0 (x0 = 0: r = b), z = d r, p = z; ||b||^2, r.r, r.z
  double v3[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int j = 0; j < RPT; ++j) {
    if (!own[j]) continue;
    const T ri = a.x_zero ? (T)bj[j] : (T)(bj[j] - wd(row_dot(j, a.x)));
    const T zi = pc ? dj[j] * ri : ri;
    rj[j] = ri;
    pj[j] = zi;
    v3[0] += bj[j] * bj[j];
    v3[1] += wd(ri) * wd(ri);
    v3[2] += wd(ri) * wd(zi);
  }
  publish(a.p, pj);  // published by the reduction's barrier
  const bool ok0 = small_reduce<3>(v3, P_init, a.bar, tgt, a.err);
  const double nb = sqrt(v3[0]), tol_abs = a.rel_tol * nb;
  double rho = v3[2];
  if (!ok0) {
    status = -1;
  } else if (v3[0] == 0.0) {  // b == 0: x = 0 after 0 iterations
#pragma unroll
    for (int j = 0; j < RPT; ++j) xj[j] = T(0);
    status = kConverged;
  } else if (sqrt(v3[1]) <= tol_abs) {
    status = kConverged;
  } else if (a.maxit <= 0) {
    status = kNotConverged;
  }
  while (status == kRun) {
    // q = A p, p.q
    T qj[RPT];
    double v1[1] = {0.0};
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      qj[j] = own[j] ? row_dot(j, a.p) : T(0);
      v1[0] += wd(pj[j]) * wd(qj[j]);
    }
    if (!small_reduce<1>(v1, P_pq, a.bar, tgt, a.err)) {
      status = -1;
      break;
    }
    const double pq = v1[0];
    if (!(pq > 0.0)) {
      status = kBreakdown;
      break;
    }
    const double alpha = rho / pq;
    const Lin<T> ax(alpha), ar(-alpha);
    double v2[2] = {0.0, 0.0};
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      if (!own[j]) continue;
      xj[j] = ax(pj[j], xj[j]);
      rj[j] = ar(qj[j], rj[j]);
      const double rw = wd(rj[j]);
      v2[0] = __fma_rn(rw, rw, v2[0]);
      v2[1] = pc ? __fma_rn(rw, wd(dj[j] * rj[j]), v2[1]) : v2[0];
    }
    if (!small_reduce<2>(v2, P_rr, a.bar, tgt, a.err)) {
      status = -1;
      break;
    }
    ++it;
    double rho_new = pc ? v2[1] : v2[0];
    if (sqrt(v2[0]) <= tol_abs) {
      if (!a.check_true) {
        status = kConverged;
        break;
      }
      // true residual t = b - A x: every block's x first
      publish(a.x, xj);
      if (!small_sync(a.bar, tgt, a.err)) {
        status = -1;
        break;
      }
      T tj[RPT];
      double vt[2] = {0.0, 0.0};
#pragma unroll
      for (int j = 0; j < RPT; ++j) {
        tj[j] = own[j] ? (T)(bj[j] - wd(row_dot(j, a.x))) : T(0);
        vt[0] += wd(tj[j]) * wd(tj[j]);
        vt[1] += wd(tj[j]) * wd(pc ? dj[j] * tj[j] : tj[j]);
      }
      if (!small_reduce<2>(vt, P_true, a.bar, tgt, a.err)) {
        status = -1;
        break;
      }
      if (sqrt(vt[0]) <= tol_abs) {
        status = kConverged;
        break;
      }
#pragma unroll
      for (int j = 0; j < RPT; ++j) rj[j] = tj[j];  // residual replacement (p is kept)
      rho_new = vt[1];
    } else if (it >= a.maxit) {
      status = kNotConverged;
      break;
    }
    const Lin<T> bp(rho_new / rho);
    rho = rho_new;
#pragma unroll
    for (int j = 0; j < RPT; ++j) pj[j] = bp(pj[j], pc ? dj[j] * rj[j] : rj[j]);
    publish(a.p, pj);
    if (!small_sync(a.bar, tgt, a.err)) {
      status = -1;
      break;
    }
  }
  publish(a.x, xj);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.c->status = status < 0 ? kNotConverged : status;
    a.c->iter = it;
    a.c->cycles = status < 0 ? 1 : 0;  // 1: a barrier timed out
  }
}

// Whether the single-launch CG serves this matrix (see above).
static bool small_cg_ok(const gko_matrix_s* A, const SolveSpec& sp) {
  if (sp.solver != 0 || sp.rel || sp.bj || A->fmt != GKO_CSR || A->plan.kind != 1 || A->n_rows <= 0 ||
      A->n_rows > kSmallRows)
    return false;
  int dev = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) !=
                                                   cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return coop != 0;
}

// Resident blocks per SM of one instantiation at the given dynamic shared
// memory (computed once per instantiation and size class).
template <typename K>
static int small_per_sm(K kern, size_t smem) {
  int nb = 0;
  if (smem > 48 * 1024 && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kSmallSmemMax) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kSmallThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

template <typename T, typename VT, int RPT>
static int small_cg_launch(const gko_matrix_s* A, SmallArgs<T, VT>& a, int G, size_t smem, bool staged,
                           cudaStream_t s) {
  void* args[] = {&a};
  if (staged) {
    auto kern = small_cg_kernel<T, VT, RPT, true>;
    // always the largest request (kSmallSmemMax), so concurrent solves with
    // different sizes never lower each other's limit
    if (smem > 48 * 1024)
      GKO_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallSmemMax));
    GKO_TRY_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)G), dim3(kSmallThreads), args, smem, s));
  } else {
    auto kern = small_cg_kernel<T, VT, RPT, false>;
    GKO_TRY_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)G), dim3(kSmallThreads), args, 0, s));
  }
  return GKO_OK;
}

template <typename T, typename VT>
static int small_cg(const gko_matrix_s* A, const double* b, T* x, bool x_zero, const SolveSpec& sp, cudaStream_t s,
                    SolveOut* out) {
  const int64_t n = A->n_rows;
  // rows per thread: the fewest (1, 2, 4) whose grid fits on the GPU at once
  int rpt = 0, G = 0;
  size_t smem = 0;
  bool staged = false;
  for (int r : {1, 2, 4}) {
    const int64_t g = (n + (int64_t)kSmallThreads * r - 1) / ((int64_t)kSmallThreads * r);
    const size_t cap = (size_t)kSmallThreads * r * (size_t)std::max(1, A->plan.max_len);
    const size_t bytes = ((cap * sizeof(int32_t) + 15) & ~(size_t)15) + cap * sizeof(VT);
    const bool st = bytes <= kSmallSmemMax;
    int per_sm = 0;
    if (r == 1) per_sm = st ? small_per_sm(small_cg_kernel<T, VT, 1, true>, bytes) : small_per_sm(small_cg_kernel<T, VT, 1, false>, 0);
    if (r == 2) per_sm = st ? small_per_sm(small_cg_kernel<T, VT, 2, true>, bytes) : small_per_sm(small_cg_kernel<T, VT, 2, false>, 0);
    if (r == 4) per_sm = st ? small_per_sm(small_cg_kernel<T, VT, 4, true>, bytes) : small_per_sm(small_cg_kernel<T, VT, 4, false>, 0);
    if (per_sm > 0 && g <= (int64_t)per_sm * sm_count()) {
      rpt = r;
      G = (int)g;
      staged = st;
      smem = st ? bytes : 0;
      break;
    }
  }
  if (!rpt) return GKO_NOT_SUPPORTED;  // the caller falls back to the multi-kernel solve
  Scratch mem;
  GKO_TRY(mem.get(sizeof(Ctl) + sizeof(T) * (size_t)n + sizeof(double) * 12 * (size_t)G + 2048, s));
  Carve cv{static_cast<char*>(mem.data())};
  Ctl* c = cv.take<Ctl>(1);
  unsigned* bar = cv.take<unsigned>(4);
  double* part = cv.take<double>(12 * (size_t)G);
  T* p = cv.take<T>(n);
  const int32_t cap32 = (int32_t)((size_t)kSmallThreads * rpt * (size_t)std::max(1, A->plan.max_len));
  SmallArgs<T, VT> a{n,  ptr<int32_t>(A->row_ptr), ptr<int32_t>(A->col), ptr<VT>(A->val),
                     b,  x, p, static_cast<const T*>(sp.minv), sp.rel_tol, sp.maxit, sp.check_true,
                     x_zero ? 1 : 0, cap32, part, bar, device_error_word(), c};
  GKO_TRY_CUDA(cudaMemsetAsync(bar, 0, 16, s));
  if (rpt == 1) GKO_TRY((small_cg_launch<T, VT, 1>(A, a, G, smem, staged, s)));
  if (rpt == 2) GKO_TRY((small_cg_launch<T, VT, 2>(A, a, G, smem, staged, s)));
  if (rpt == 4) GKO_TRY((small_cg_launch<T, VT, 4>(A, a, G, smem, staged, s)));
  Ctl* hc = host_ctl();
  GKO_TRY(read_ctl(c, hc, s));
  if (hc->cycles) return fail(GKO_TIMEOUT, "single-launch CG: a grid barrier wait timed out");
  out->status = hc->status;
  out->iterations = hc->iter;
  out->cycles = 0;
  return GKO_OK;
}

// ------------------------------------------------ cluster CG (tiny n) --
//
// The same CG as small_cg_kernel (Saad Alg. 6.18 / 9.1, true-residual check,
// residual replacement, breakdown and iteration-cap rules) for n <= 16 x 256
// x 4 rows, run by ONE thread-block cluster of CS <= 16 CTAs instead of a
// cooperative grid: CTA k owns rows [k RB, (k+1) RB) (RB = 256 RPT) and keeps
// its slice of p (and, for the true-residual check, of x) in shared memory;
// the SpMV gathers p from the owning CTA's shared memory through distributed
// shared memory, and every grid barrier becomes a hardware cluster barrier
// (barrier.cluster with release/acquire semantics) instead of a round trip
// through an L2 counter.  Reductions: each CTA publishes its block sums in
// its shared memory, and after the barrier warp 0 of every CTA reads the CS
// partials (lane l from CTA l) and adds them with a fixed butterfly, so all
// CTAs hold bit-identical totals and take the same branch.  That uniformity is
// what keeps the hardware barriers safe: no CTA leaves the loop or the kernel
// on its own, and a last barrier keeps every CTA's shared memory alive until
// the others have finished reading it.  It serves FP64 solves; the FP32 /
// BF16 inner solves of mixed precision keep the cooperative-grid kernel.
namespace cgx = cooperative_groups;
constexpr int kClusterMax = 16;

// Cluster barrier and distributed-shared-memory loads as inline PTX with
// memory clobbers, so the compiler can move no shared-memory access across
// the barrier and no remote load ahead of it (built on the cooperative-groups
// calls, one instantiation read a remote reduction slot before its owner had
// written it).  Call the barrier from control flow that is the same in every
// thread of the cluster.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ uint32_t dsmem_addr(const void* local, unsigned rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ double dsmem_ld(const double* local, unsigned rank) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(dsmem_addr(local, rank)) : "memory");
  return v;
}
__device__ __forceinline__ float dsmem_ld(const float* local, unsigned rank) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(dsmem_addr(local, rank)) : "memory");
  return v;
}
constexpr int64_t kClusterRows = (int64_t)kClusterMax * kSmallThreads * 4;
constexpr size_t kClusterSmemMax = 200 * 1024;

template <int NV>
__device__ __forceinline__ void cluster_reduce(const cgx::cluster_group& cl, double (&v)[NV], double (*s_red)[4],
                                               int site, double* s_tot) {
  block_sum_n<kSmallThreads, NV>(v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) s_red[site][k] = v[k];
  cluster_barrier();
  if (threadIdx.x < 32) {
    const int cs = (int)cl.num_blocks();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = (int)threadIdx.x < cs ? dsmem_ld(&s_red[site][k], threadIdx.x) : 0.0;
      t = subwarp_sum<32>(t, 0xffffffffu);
      if (threadIdx.x == 0) s_tot[k] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = s_tot[k];
}

template <typename T, typename VT, int RPT, bool SMEM>
__global__ void __launch_bounds__(kSmallThreads) cluster_cg_kernel(SmallArgs<T, VT> a) {
  using AT = acc_t<VT>;
  constexpr int RB = kSmallThreads * RPT;
  const cgx::cluster_group cl = cgx::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s_p = reinterpret_cast<T*>(smem_raw);
  T* s_x = s_p + RB;
  int32_t* scol = reinterpret_cast<int32_t*>(smem_raw + 2 * (size_t)RB * sizeof(T));
  VT* sval = reinterpret_cast<VT*>(reinterpret_cast<unsigned char*>(scol) +
                                   (((size_t)a.block_cap * sizeof(int32_t) + 15) & ~(size_t)15));
  __shared__ double s_red[4][4];
  __shared__ double s_tot[4];
  const int64_t row0 = (int64_t)rank * RB;
  const int64_t row1 = row0 + RB < a.n ? row0 + RB : a.n;
  const int32_t e0 = __ldg(a.rp + row0), e1 = __ldg(a.rp + row1);
  if (SMEM) {
    for (int32_t k = e0 + (int32_t)threadIdx.x; k < e1; k += kSmallThreads) {
      scol[k - e0] = __ldg(a.col + k);
      sval[k - e0] = a.val[k];
    }
  }
  int32_t ks[RPT], ke[RPT];
  bool own[RPT];
  double bj[RPT];
  T xj[RPT], rj[RPT], pj[RPT], dj[RPT];
#pragma unroll
  for (int j = 0; j < RPT; ++j) {
    const int64_t i = row0 + threadIdx.x + (int64_t)j * kSmallThreads;
    own[j] = i < a.n;
    ks[j] = own[j] ? __ldg(a.rp + i) - (SMEM ? e0 : 0) : 0;
    ke[j] = own[j] ? __ldg(a.rp + i + 1) - (SMEM ? e0 : 0) : 0;
    bj[j] = own[j] ? a.b[i] : 0.0;
    xj[j] = own[j] && !a.x_zero ? a.x[i] : T(0);
    dj[j] = own[j] && a.d ? a.d[i] : T(1);
  }
  const bool pc = a.d != nullptr;
  // element c of a vector whose slices live in the CTAs' shared memory (s)
  auto gat = [&](const T* s, int32_t c) -> T {
    const int owner = c / RB, off = c - owner * RB;
    return owner == rank ? s[off] : dsmem_ld(s + off, (unsigned)owner);
  };
  // row j of A v, v in the CTAs' slices s; up to 8 gathers issued before their FMAs
  auto row_dot = [&](int j, const T* s) -> T {
    constexpr int U = 8;
    AT acc = AT(0);
    for (int32_t k = ks[j]; k < ke[j]; k += U) {
      VT w[U];
      T g[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool in = k + u < ke[j];
        const int32_t c = in ? (SMEM ? scol[k + u] : __ldg(a.col + k + u)) : 0;
        w[u] = in ? (SMEM ? sval[k + u] : a.val[k + u]) : VT(0);
        g[u] = in ? gat(s, c) : T(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (k + u < ke[j]) acc = madd(to_acc(w[u]), to_acc(g[u]), acc);
    }
    return (T)acc;
  };
  auto publish = [&](T* dst, const T (&v)[RPT]) {
#pragma unroll
    for (int j = 0; j < RPT; ++j)
      if (own[j]) dst[threadIdx.x + j * kSmallThreads] = v[j];
  };
  int status = kRun, it = 0;
  // r = b - A x0 (x0 = 0: r = b), z = d r, p = z; ||b||^2, r.r, r.z
  if (!a.x_zero) {
    publish(s_x, xj);
    cluster_barrier();
  } else {
    __syncthreads();  // the staged entries
  }
  double v3[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int j = 0; j < RPT; ++j) {
    if (!own[j]) continue;
    const T ri = a.x_zero ? (T)bj[j] : (T)(bj[j] - wd(row_dot(j, s_x)));
    const T zi = pc ? dj[j] * ri : ri;
    rj[j] = ri;
    pj[j] = zi;
    v3[0] += bj[j] * bj[j];
    v3[1] += wd(ri) * wd(ri);
    v3[2] += wd(ri) * wd(zi);
  }
  publish(s_p, pj);  // visible after the reduction's cluster barrier
  cluster_reduce<3>(cl, v3, s_red, 0, s_tot);
  const double nb = sqrt(v3[0]), tol_abs = a.rel_tol * nb;
  double rho = v3[2];
  if (v3[0] == 0.0) {  // b == 0: x = 0 after 0 iterations
#pragma unroll
    for (int j = 0; j < RPT; ++j) xj[j] = T(0);
    status = kConverged;
  } else if (sqrt(v3[1]) <= tol_abs) {
    status = kConverged;
  } else if (a.maxit <= 0) {
    status = kNotConverged;
  }
  while (status == kRun) {
    T qj[RPT];
    double v1[1] = {0.0};
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      qj[j] = own[j] ? row_dot(j, s_p) : T(0);
      v1[0] += wd(pj[j]) * wd(qj[j]);
    }
    cluster_reduce<1>(cl, v1, s_red, 1, s_tot);
    const double pq = v1[0];
    if (!(pq > 0.0)) {
      status = kBreakdown;
      break;
    }
    const double alpha = rho / pq;
    const Lin<T> ax(alpha), ar(-alpha);
    double v2[2] = {0.0, 0.0};
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      if (!own[j]) continue;
      xj[j] = ax(pj[j], xj[j]);
      rj[j] = ar(qj[j], rj[j]);
      const double rw = wd(rj[j]);
      v2[0] = __fma_rn(rw, rw, v2[0]);
      v2[1] = pc ? __fma_rn(rw, wd(dj[j] * rj[j]), v2[1]) : v2[0];
    }
    cluster_reduce<2>(cl, v2, s_red, 2, s_tot);
    ++it;
    double rho_new = pc ? v2[1] : v2[0];
    if (sqrt(v2[0]) <= tol_abs) {
      if (!a.check_true) {
        status = kConverged;
        break;
      }
      // true residual t = b - A x: every CTA's slice of x first
      publish(s_x, xj);
      cluster_barrier();
      T tj[RPT];
      double vt[2] = {0.0, 0.0};
#pragma unroll
      for (int j = 0; j < RPT; ++j) {
        tj[j] = own[j] ? (T)(bj[j] - wd(row_dot(j, s_x))) : T(0);
        vt[0] += wd(tj[j]) * wd(tj[j]);
        vt[1] += wd(tj[j]) * wd(pc ? dj[j] * tj[j] : tj[j]);
      }
      cluster_reduce<2>(cl, vt, s_red, 3, s_tot);
      if (sqrt(vt[0]) <= tol_abs) {
        status = kConverged;
        break;
      }
#pragma unroll
      for (int j = 0; j < RPT; ++j) rj[j] = tj[j];  // residual replacement (p is kept)
      rho_new = vt[1];
    } else if (it >= a.maxit) {
      status = kNotConverged;
      break;
    }
    const Lin<T> bp(rho_new / rho);
    rho = rho_new;
#pragma unroll
    for (int j = 0; j < RPT; ++j) pj[j] = bp(pj[j], pc ? dj[j] * rj[j] : rj[j]);
    publish(s_p, pj);
    cluster_barrier();
  }
#pragma unroll
  for (int j = 0; j < RPT; ++j)
    if (own[j]) a.x[row0 + threadIdx.x + (int64_t)j * kSmallThreads] = xj[j];
  if (rank == 0 && threadIdx.x == 0) {
    a.c->status = status;
    a.c->iter = it;
    a.c->cycles = 0;
  }
  cluster_barrier();  // no CTA's shared memory goes while another may still read it
}

// Launch the cluster CG when it applies (n <= kClusterRows and a cluster of
// the needed size fits); GKO_NOT_SUPPORTED otherwise (the caller takes the
// cooperative-grid kernel).
template <typename T, typename VT, int RPT>
static int cluster_cg_launch(SmallArgs<T, VT>& a, int CS, size_t smem, bool staged, cudaStream_t s) {
  auto kern = staged ? cluster_cg_kernel<T, VT, RPT, true> : cluster_cg_kernel<T, VT, RPT, false>;
  // attributes set once per instantiation, to the largest request, so
  // concurrent solves (serving threads) never undo each other's setting
  static const bool attrs_ok = [] {
    bool ok = true;
    for (auto k : {cluster_cg_kernel<T, VT, RPT, true>, cluster_cg_kernel<T, VT, RPT, false>})
      ok = ok && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
           cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClusterSmemMax) ==
               cudaSuccess;
    if (!ok) cudaGetLastError();
    return ok;
  }();
  if (!attrs_ok || smem > kClusterSmemMax) return GKO_NOT_SUPPORTED;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)CS);
  cfg.blockDim = dim3(kSmallThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return GKO_NOT_SUPPORTED;
  }
  GKO_TRY_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
  return GKO_OK;
}

template <typename T, typename VT>
static int cluster_cg(const gko_matrix_s* A, const double* b, T* x, bool x_zero, const SolveSpec& sp,
                      cudaStream_t s, SolveOut* out) {
  const int64_t n = A->n_rows;
  if (n > kClusterRows) return GKO_NOT_SUPPORTED;
  // rows per thread: the fewest (1, 2, 4) for which 16 CTAs cover n
  int rpt = 1;
  while (rpt < 4 && n > (int64_t)kClusterMax * kSmallThreads * rpt) rpt *= 2;
  const int64_t RB = (int64_t)kSmallThreads * rpt;
  const int CS = (int)((n + RB - 1) / RB);
  const size_t cap = (size_t)RB * (size_t)std::max(1, A->plan.max_len);
  const size_t vec = 2 * (size_t)RB * sizeof(T);
  const size_t stage = ((cap * sizeof(int32_t) + 15) & ~(size_t)15) + cap * sizeof(VT);
  const bool staged = vec + stage <= kClusterSmemMax;
  const size_t smem = staged ? vec + stage : vec;
  Scratch mem;
  GKO_TRY(mem.get(sizeof(Ctl) + 1024, s));
  Carve cv{static_cast<char*>(mem.data())};
  Ctl* c = cv.take<Ctl>(1);
  SmallArgs<T, VT> a{n,  ptr<int32_t>(A->row_ptr), ptr<int32_t>(A->col), ptr<VT>(A->val),
                     b,  x, nullptr, static_cast<const T*>(sp.minv), sp.rel_tol, sp.maxit, sp.check_true,
                     x_zero ? 1 : 0, (int32_t)cap, nullptr, nullptr, device_error_word(), c};
  int rc = GKO_NOT_SUPPORTED;
  if (rpt == 1) rc = cluster_cg_launch<T, VT, 1>(a, CS, smem, staged, s);
  if (rpt == 2) rc = cluster_cg_launch<T, VT, 2>(a, CS, smem, staged, s);
  if (rpt == 4) rc = cluster_cg_launch<T, VT, 4>(a, CS, smem, staged, s);
  if (rc != GKO_OK) return rc;
  Ctl* hc = host_ctl();
  GKO_TRY(read_ctl(c, hc, s));
  out->status = hc->status;
  out->iterations = hc->iter;
  out->cycles = 0;
  return GKO_OK;
}

// One Krylov solve on the device.  A: matrix whose value type matches T
// (double: F64; float: F32/BF16).  b: FP64 right-hand side; x: T vector,
// x0 on entry (x_zero: treat x0 as zero without reading it).
template <typename T>
static int krylov_core(const gko_matrix_s* A, const double* b, T* x, bool x_zero, const SolveSpec& sp,
                       cudaStream_t s, SolveOut* out) {
  if (small_cg_ok(A, sp)) {
    int rc = GKO_NOT_SUPPORTED;
    if constexpr (std::is_same<T, double>::value) {
      if (A->dtype == GKO_F64) rc = cluster_cg<double, double>(A, b, x, x_zero, sp, s, out);
      if (rc == GKO_NOT_SUPPORTED && A->dtype == GKO_F64) rc = small_cg<double, double>(A, b, x, x_zero, sp, s, out);
    } else {
      // FP32 / BF16 inner solves keep the cooperative-grid kernel (see
      // cluster_cg_kernel)
      if (A->dtype == GKO_F32) rc = small_cg<float, float>(A, b, x, x_zero, sp, s, out);
      if (A->dtype == GKO_BF16) rc = small_cg<float, __nv_bfloat16>(A, b, x, x_zero, sp, s, out);
    }
    if (rc != GKO_NOT_SUPPORTED) return rc;
  }
  const int64_t n = A->n_rows;
  const int m = std::max(1, sp.restart);
  const int nvec = sp.solver == 0 ? (sp.bj ? 4 : 3) : sp.solver == 1 ? 9 : (m + 2);
  const T* dinv = static_cast<const T*>(sp.minv);
  const T* bj = static_cast<const T*>(sp.bj);  // block-Jacobi inverse blocks
  const int bs = sp.bs;
  const size_t spmv_sb = spmv_scratch_bytes(A);
  const size_t bytes = 256 * 16 + sizeof(Ctl) + sizeof(double) * 3 * kDotSlots + 512 +
                       (size_t)nvec * (sizeof(T) * ((size_t)n + 64) + 320) + spmv_sb + 320 +
                       sizeof(double) * ((size_t)(m + 1) * m + 6 * (m + 2) + (size_t)(m + 1) * kMultiSlots) + 4096;
  Scratch mem;
  GKO_TRY(mem.get(bytes, s));
  Carve cv{static_cast<char*>(mem.data())};
  Ctl* c = cv.take<Ctl>(1);
  unsigned* counter = cv.take<unsigned>(4);
  double* partials = cv.take<double>(3 * kDotSlots);  // up to 3 sums per block
  void* spmv_scratch = spmv_sb ? cv.take<char>(spmv_sb) : nullptr;
  RedWs ws{partials, counter};
  GKO_TRY_CUDA(cudaMemsetAsync(counter, 0, 16, s));
  Ctl init{};
  init.maxit = sp.maxit;
  init.check_true = sp.check_true;
  init.delta = sp.rel ? sp.rel->delta : 0.0;
  GKO_TRY_CUDA(cudaMemcpyAsync(c, &init, sizeof(Ctl), cudaMemcpyHostToDevice, s));
  Ctl* hc = host_ctl();
  const int vg = vec_grid(n), rg = reduce_grid(n);
  const bool fused = spmv_fuses_dot(A);
  auto spmv = [&](const T* in, T* outv, const T* w, const int* gate, bool want_yy = false) -> int {
    if (w && fused) {
      DotSpec d;
      d.w = w;
      d.want_yy = want_yy ? 1 : 0;
      d.partials = partials;
      d.counter = counter;
      d.result = c->red;
      return spmv_run(A, in, outv, 1.0, 0.0, s, spmv_scratch, &d, gate);
    }
    GKO_TRY(spmv_run(A, in, outv, 1.0, 0.0, s, spmv_scratch, nullptr, gate));
    if (w) GKO_TRY_CUDA(launch_k(dot2_kernel<T>, dim3(rg), dim3(256), 0, s, n, w, outv, ws, c->red, gate));
    return GKO_OK;
  };
  out->iterations = 0;
  out->cycles = 0;

  if (sp.solver == 0 || sp.solver == 1) {
    T* r = cv.take<T>(n);
    T* p = cv.take<T>(n);
    T* q = cv.take<T>(n);
    T *rh = nullptr, *v = nullptr, *sv = nullptr, *tv = nullptr, *ph = nullptr, *sh = nullptr;
    T* zb = (sp.solver == 0 && bj) ? cv.take<T>(n) : nullptr;  // CG with block-Jacobi: z = M^-1 r
    if (sp.solver == 1) {
      rh = cv.take<T>(n);
      v = cv.take<T>(n);
      sv = cv.take<T>(n);
      tv = cv.take<T>(n);
      if (dinv || bj) {
        ph = cv.take<T>(n);
        sh = cv.take<T>(n);
      }
    }
    if (!x_zero) GKO_TRY(spmv(x, q, nullptr, nullptr));
    if (sp.solver == 0 && bj) {
      // z = M^-1 r, p = z, rho = r.z
      init_residual_kernel<T><<<rg, 256, 0, s>>>(n, b, x_zero ? nullptr : q, r, nullptr, nullptr, nullptr, nullptr,
                                                 ws, InitOp{c, sp.rel_tol, 0});
      GKO_TRY_CUDA(bj_launch<T>(dim3(rg), s, n, bs, bj, (const T*)r, zb, p, ws, BjInitOp{c}, &c->done, nullptr));
    } else if (sp.solver == 0)
      init_residual_kernel<T><<<rg, 256, 0, s>>>(n, b, x_zero ? nullptr : q, r, p, nullptr, nullptr, nullptr, ws,
                                                 InitOp{c, sp.rel_tol, 0}, dinv);
    else
      init_residual_kernel<T><<<rg, 256, 0, s>>>(n, b, x_zero ? nullptr : q, r, rh, nullptr, p, v, ws,
                                                 InitOp{c, sp.rel_tol, 1});
    GKO_TRY_CUDA(cudaGetLastError());
    if (x_zero) zero_kernel<T><<<vg, 256, 0, s>>>(n, x);
    GKO_TRY(read_ctl(c, hc, s));
    if (hc->nb == 0.0) zero_kernel<T><<<vg, 256, 0, s>>>(n, x);
    if (!hc->done && sp.maxit <= 0) {  // no iterations allowed
      hc->status = kNotConverged;
      hc->done = 1;
    }
    // An iteration's kernels run back to back on s: each is launched with
    // programmatic serialization (PdlScope), so its dispatch overlaps the
    // drain of the one before; each waits for that one before touching memory.
    const dim3 B256(256);
    auto enqueue = [&](int count) -> int {
      PdlScope pdl(true);
      for (int it = 0; it < count; ++it) {
        if (sp.solver == 0) {
          GKO_TRY(spmv(p, q, p, &c->done));
          if (bj) {
            GKO_TRY_CUDA(launch_k(cg_update_kernel<T, false, true>, dim3(rg), B256, 0, s, n, x, r, p, q, c, ws,
                                  (const T*)nullptr));
            GKO_TRY_CUDA(bj_launch<T>(dim3(rg), s, n, bs, bj, (const T*)r, zb, (T*)nullptr, ws, BjStepOp{c},
                                      (const int*)&c->done, (const int*)nullptr));
            GKO_TRY_CUDA(launch_k(cg_p_kernel<T, false>, dim3(vg), B256, 0, s, n, (const T*)zb, p, c,
                                  (const T*)nullptr));
          } else if (dinv) {
            GKO_TRY_CUDA(launch_k(cg_update_kernel<T, true>, dim3(rg), B256, 0, s, n, x, r, p, q, c, ws, dinv));
            GKO_TRY_CUDA(launch_k(cg_p_kernel<T, true>, dim3(vg), B256, 0, s, n, r, p, c, dinv));
          } else {
            GKO_TRY_CUDA(launch_k(cg_update_kernel<T, false>, dim3(rg), B256, 0, s, n, x, r, p, q, c, ws,
                                  (const T*)nullptr));
            GKO_TRY_CUDA(launch_k(cg_p_kernel<T, false>, dim3(vg), B256, 0, s, n, r, p, c, (const T*)nullptr));
          }
        } else if (bj) {
          // right preconditioned: ph = M^-1 p, sh = M^-1 s
          GKO_TRY_CUDA(launch_k(bicg_p_kernel<T>, dim3(vg), B256, 0, s, n, (const T*)r, p, (const T*)v, c,
                                (const T*)nullptr, (T*)nullptr));
          GKO_TRY_CUDA(bj_launch<T>(dim3(vg), s, n, bs, bj, (const T*)p, ph, (T*)nullptr, ws, NoOp{},
                                    (const int*)&c->done, (const int*)nullptr));
          GKO_TRY(spmv(ph, v, rh, &c->done));
          GKO_TRY_CUDA(launch_k(bicg_s_kernel<T>, dim3(rg), B256, 0, s, n, (const T*)r, (const T*)v, sv, c, ws,
                                (const T*)nullptr, (T*)nullptr));
          GKO_TRY_CUDA(bj_launch<T>(dim3(vg), s, n, bs, bj, (const T*)sv, sh, (T*)nullptr, ws, NoOp{},
                                    (const int*)&c->phase, (const int*)nullptr));
          GKO_TRY(spmv(sh, tv, sv, &c->phase, true));
          GKO_TRY_CUDA(launch_k(bicg_x_kernel<T>, dim3(rg), B256, 0, s, n, x, (const T*)p, (const T*)sv,
                                (const T*)tv, r, (const T*)rh, c, ws, (const T*)ph, (const T*)sh));
        } else {
          GKO_TRY_CUDA(launch_k(bicg_p_kernel<T>, dim3(vg), B256, 0, s, n, r, p, v, c, dinv, ph));
          GKO_TRY(spmv(dinv ? ph : p, v, rh, &c->done));
          GKO_TRY_CUDA(launch_k(bicg_s_kernel<T>, dim3(rg), B256, 0, s, n, r, v, sv, c, ws, dinv, sh));
          GKO_TRY(spmv(dinv ? sh : sv, tv, sv, &c->phase, true));
          GKO_TRY_CUDA(launch_k(bicg_x_kernel<T>, dim3(rg), B256, 0, s, n, x, p, sv, tv, r, rh, c, ws,
                                (const T*)ph, (const T*)sh));
        }
      }
      return GKO_OK;
    };
    // the first batch launches directly (it also initialises the launch
    // configuration caches); later batches replay one captured graph
    // reliable updates stop a batch early (its remaining kernels run gated
    // off), so they poll every 8 iterations (BiCGSTAB on 128^3: 85 ms at 8,
    // 89 ms at 16, 102 ms at 32)
    const int graph_iters = sp.check_every > 0 ? sp.check_every : sp.rel ? 8 : kGraphIters;
    BatchGraph graph;
    bool first = true;
    while (!hc->done) {
      if (first || graph.refused) {
        GKO_TRY(enqueue(first && sp.check_every <= 0 ? 8 : graph_iters));
        first = false;
      } else {
        if (!graph.e) GKO_TRY(graph.capture(s, [&] { return enqueue(graph_iters); }));
        if (graph.e)
          GKO_TRY_CUDA(cudaGraphLaunch(graph.e, s));
        else
          GKO_TRY(enqueue(graph_iters));
      }
      GKO_TRY(read_ctl(c, hc, s));
      if (hc->status == kCheck && sp.rel) {
        if constexpr (std::is_same<T, float>::value) {
          // reliable update: fold d into the FP64 x, replace r by b - A64 x
          const RelSpec& rl = *sp.rel;
          fold_kernel<<<vg, 256, 0, s>>>(n, rl.x64, x);
          GKO_TRY_CUDA(cudaGetLastError());
          GKO_TRY(spmv_run(rl.A64, rl.x64, rl.q64, 1.0, 0.0, s, rl.scratch, nullptr, nullptr));
          const bool half = sp.solver == 1 && hc->half;
          T* dst = (sp.solver == 1 && !half) ? r : q;
          rel_replace_kernel<T><<<rg, 256, 0, s>>>(n, rl.b64, rl.q64, dst, sp.solver == 1 ? rh : nullptr,
                                                   sp.solver == 0 ? dinv : nullptr, ws,
                                                   RelOp{c, sp.solver, half ? 1 : 0});
          if (sp.solver == 0 && bj) {
            // z = M^-1 t and rho_new = t.z for the replaced residual t
            GKO_TRY_CUDA(bj_launch<T>(dim3(rg), s, n, bs, bj, (const T*)q, zb, (T*)nullptr, ws, BjReplaceOp{c},
                                      (const int*)nullptr, (const int*)&c->replace));
            cg_replace_kernel<T><<<rg, 256, 0, s>>>(n, r, p, q, c, ws, nullptr, zb);
          } else if (sp.solver == 0)
            cg_replace_kernel<T><<<rg, 256, 0, s>>>(n, r, p, q, c, ws, dinv);
          else if (half)
            bicg_restart_kernel<T><<<rg, 256, 0, s>>>(n, r, rh, p, v, q, c, ws);
          GKO_TRY_CUDA(cudaGetLastError());
          out->cycles += 1;
          GKO_TRY(read_ctl(c, hc, s));
        }
      } else if (hc->status == kCheck) {  // verify with the true residual
        GKO_TRY(spmv(x, q, nullptr, nullptr));
        true_res_kernel<T><<<rg, 256, 0, s>>>(n, b, q, ws, TrueResOp{c}, sp.solver == 0 ? dinv : nullptr);
        if (sp.solver == 0 && bj) {
          // z = M^-1 t and rho_new = t.z for the replaced residual t
          GKO_TRY_CUDA(bj_launch<T>(dim3(rg), s, n, bs, bj, (const T*)q, zb, (T*)nullptr, ws, BjReplaceOp{c},
                                    (const int*)nullptr, (const int*)&c->replace));
          cg_replace_kernel<T><<<rg, 256, 0, s>>>(n, r, p, q, c, ws, nullptr, zb);
        } else if (sp.solver == 0)
          cg_replace_kernel<T><<<rg, 256, 0, s>>>(n, r, p, q, c, ws, dinv);
        else
          bicg_restart_kernel<T><<<rg, 256, 0, s>>>(n, r, rh, p, v, q, c, ws);
        GKO_TRY_CUDA(cudaGetLastError());
        GKO_TRY(read_ctl(c, hc, s));
      }
    }
    if constexpr (std::is_same<T, float>::value) {
      if (sp.rel) {  // what the recurrences moved since the last update
        fold_kernel<<<vg, 256, 0, s>>>(n, sp.rel->x64, x);
        GKO_TRY_CUDA(cudaGetLastError());
      }
    }
  } else {
    const int64_t ld = ((int64_t)n + 63) / 64 * 64;
    T* V = cv.take<T>((size_t)ld * (m + 1));
    T* w = cv.take<T>(n);
    double* H = cv.take<double>((size_t)(m + 1) * m);
    double* cs = cv.take<double>(m + 1);
    double* sn = cv.take<double>(m + 1);
    double* g = cv.take<double>(m + 2);
    double* h1 = cv.take<double>(m + 2);
    double* h2 = cv.take<double>(m + 2);
    double* ny = cv.take<double>(m + 2);
    double* mpart = cv.take<double>((size_t)(m + 1) * kMultiSlots);
    // ||b|| and the zero-b case through the common init kernel
    init_residual_kernel<T><<<rg, 256, 0, s>>>(n, b, nullptr, w, nullptr, nullptr, nullptr, nullptr, ws,
                                               InitOp{c, sp.rel_tol, 2});
    if (x_zero) zero_kernel<T><<<vg, 256, 0, s>>>(n, x);
    GKO_TRY_CUDA(cudaGetLastError());
    GKO_TRY(read_ctl(c, hc, s));
    if (hc->nb == 0.0) {
      zero_kernel<T><<<vg, 256, 0, s>>>(n, x);
    } else {
      // the initial residual decides afresh in the first cycle start (done =
      // 0, status = kRun = 0; set on the device, no host source to outlive)
      static_assert(kRun == 0, "kRun is written as a zero word");
      GKO_TRY_CUDA(cudaMemsetAsync(&c->done, 0, sizeof(int), s));
      GKO_TRY_CUDA(cudaMemsetAsync(&c->status, 0, sizeof(int), s));
      hc->done = 0;
    }
    int64_t mg = std::max<int64_t>(1, std::min<int64_t>((n + 2047) / 2048, kMultiSlots));
    bool first = true;
    while (!hc->done) {
      // cycle start: v0 = b - A x
      if (!(first && x_zero)) GKO_TRY(spmv(x, w, nullptr, &c->done));
      gm_start_kernel<T><<<rg, 256, 0, s>>>(n, b, (first && x_zero) ? nullptr : w, V, c, ws, GmStartOp{c, g, m});
      first = false;
      if (hc->iter >= sp.maxit) {
        // iteration cap reached: this start only decides the final status
        // (converged or not) and always ends the solve, so the cycle's
        // Arnoldi steps are not launched (gated, they still cost about 270
        // launches: 2.5 ms per call at n = 2.1M)
        GKO_TRY_CUDA(cudaGetLastError());
        GKO_TRY(read_ctl(c, hc, s));
        continue;
      }
      gm_scale_kernel<T><<<vg, 256, 0, s>>>(n, V, &c->beta, c);
      for (int j = 0; j < m; ++j) {
        PdlScope pdl(true);  // as in the CG / BiCGSTAB iterations
        T* vj = V + (int64_t)j * ld;
        // w = A v_j with ||w||^2 from the SpMV epilogue (red[0])
        GKO_TRY(spmv(vj, w, w, &c->phase));
        // classical Gram-Schmidt; the second pass runs only when the first
        // shrank ||w|| below ||w0|| / sqrt(2) (selective reorthogonalisation)
        for (int pass = 0; pass < 2; ++pass) {
          double* hp = pass == 0 ? h1 : h2;
          GKO_TRY_CUDA(launch_k(gm_multidot_kernel<T>, dim3((unsigned)mg, (unsigned)(j + 1)), dim3(256), 0, s, n,
                                (const T*)V, ld, (const T*)w, mpart, c, pass));
          GKO_TRY_CUDA(launch_k(gm_multidot_finish_kernel, dim3(j + 1), dim3(256), 0, s, (int)mg,
                                (const double*)mpart, hp, 0, c, pass));
          GKO_TRY_CUDA(launch_k(gm_axpy_kernel<T, true>, dim3(rg), dim3(256), 0, s, n, j + 1, (const double*)hp,
                                (const T*)V, ld, w, c, ws, pass));
        }
        GKO_TRY_CUDA(launch_k(gm_givens_kernel, dim3(1), dim3(1), 0, s, j, m, (const double*)h1, (const double*)h2, H,
                              cs, sn, g, c));
        if (j + 1 <= m)
          GKO_TRY_CUDA(launch_k(gm_next_kernel<T>, dim3(vg), dim3(256), 0, s, n, (const T*)w,
                                V + (int64_t)(j + 1) * ld, c));
      }
      gm_backsolve_kernel<<<1, 1, 0, s>>>(m, H, g, ny, c);
      gm_update_x_kernel<T><<<vg, 256, 0, s>>>(n, ny, V, ld, x, c);
      gm_close_kernel<<<1, 1, 0, s>>>(c);
      GKO_TRY_CUDA(cudaGetLastError());
      GKO_TRY(read_ctl(c, hc, s));
    }
  }
  out->status = hc->status;
  out->iterations = hc->iter;
  if (sp.solver == 2) out->cycles = hc->cycles;  // CG / BiCGSTAB: reliable updates counted above
  return GKO_OK;
}

// true relative residual ||b - A x|| / ||b|| in FP64 (A: F64)
static int true_rel_residual(const gko_matrix_s* A, const double* b, const double* x, double nb, double* out,
                             cudaStream_t s) {
  const int64_t n = A->n_rows;
  if (nb == 0.0) {
    *out = 0.0;
    return GKO_OK;
  }
  Scratch mem;
  const size_t sb = spmv_scratch_bytes(A);
  GKO_TRY(mem.get(sizeof(double) * (n + 2 * kDotSlots) + sizeof(Ctl) + sb + 2048, s));
  Carve cv{static_cast<char*>(mem.data())};
  Ctl* c = cv.take<Ctl>(1);
  unsigned* counter = cv.take<unsigned>(4);
  double* partials = cv.take<double>(2 * kDotSlots);
  double* q = cv.take<double>(n);
  void* ss = sb ? cv.take<char>(sb) : nullptr;
  GKO_TRY_CUDA(cudaMemsetAsync(counter, 0, 16, s));
  GKO_TRY(spmv_run(A, x, q, 1.0, 0.0, s, ss, nullptr, nullptr));
  final_res_kernel<double><<<reduce_grid(n), 256, 0, s>>>(n, b, q, RedWs{partials, counter}, c);
  GKO_TRY_CUDA(cudaGetLastError());
  double rr = 0.0;
  GKO_TRY_CUDA(cudaMemcpyAsync(&rr, &c->rr, sizeof(double), cudaMemcpyDeviceToHost, s));
  GKO_TRY_CUDA(cudaStreamSynchronize(s));
  *out = sqrt(rr) / nb;
  return GKO_OK;
}

static int map_status(int st) {
  switch (st) {
    case kConverged: return GKO_OK;
    case kBreakdown: return GKO_BREAKDOWN;
    default: return GKO_NOT_CONVERGED;
  }
}

// Low-precision copy of A cached on the handle for mixed-precision solves.
// A large CSR matrix whose rows are nearly equal in length (ELL padding at
// most kInnerEllFill x nnz: stencils) gets its copy in ELL: with 4-byte values
// the column-major ELL kernel streams the operator faster than the CSR
// kernels (7-point 128^3 FP32 SpMV 30 us vs 41 us), while in FP64 the CSR
// row-block kernel keeps up (CG on 7-point 256^3: 302 ms CSR, 314 ms ELL).
// Systems small enough for the single-launch CG (CSR only) keep CSR.
constexpr double kInnerEllFill = 1.2;
static int lowp_copy(gko_matrix A, gko_dtype to, cudaStream_t s, gko_matrix* out) {
  std::lock_guard<std::mutex> lk(A->mu);
  auto it = A->lowp.find((int)to);
  if (it != A->lowp.end()) {
    *out = it->second;
    return GKO_OK;
  }
  gko_matrix m = nullptr;
  if (A->fmt == GKO_CSR && A->n_rows > kSmallRows) {
    gko_matrix e = nullptr;
    const int rc = gko_matrix_convert_to_ell(A, kInnerEllFill, s, &e);
    if (rc == GKO_OK) {
      const int rc2 = gko_matrix_convert_values(e, to, s, &m);
      gko_matrix_destroy(e);
      GKO_TRY(rc2);
    } else if (rc != GKO_FORMAT_UNSUITABLE) {
      return rc;
    }
  }
  if (!m) GKO_TRY(gko_matrix_convert_values(A, to, s, &m));
  A->lowp[(int)to] = m;
  *out = m;
  return GKO_OK;
}

static int norm2_host(const double* v, int64_t n, double* out, cudaStream_t s) {
  double d = 0.0;
  GKO_TRY(gko_dot(n, v, v, &d, s));
  *out = sqrt(d);
  return GKO_OK;
}

// r = b - A x (FP64)
__global__ void residual64_kernel(int64_t n, const double* __restrict__ b, double* __restrict__ q) {
  GKO_GRID_LOOP(i, n) q[i] = b[i] - q[i];
}

static int solve_entry(int solver, gko_matrix A, const double* b, double* x, double rel_tol, int32_t max_iters,
                       const gko_solve_opts* opts, gko_solve_result* res, void* stream) {
  if (!A || !res) return fail(GKO_INVALID_ARG, "null matrix or result");
  res->status = GKO_NOT_CONVERGED;
  res->iterations = res->outer_iterations = 0;
  res->rel_residual = 0.0;
  if (A->n_rows != A->n_cols) return fail(GKO_INVALID_ARG, "solvers need a square matrix");
  if (A->dtype != GKO_F64) return fail(GKO_INVALID_ARG, "solvers take the FP64 matrix (mixed precision copies it)");
  if (A->n_rows > 0 && (!b || !x)) return fail(GKO_INVALID_ARG, "null b or x");
  if (!(rel_tol >= 0.0) || max_iters < 0) return fail(GKO_INVALID_ARG, "bad tolerance or iteration cap");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = A->n_rows;
  if (n == 0) {
    res->status = GKO_OK;
    return GKO_OK;
  }
  gko_solve_opts o{};
  if (opts) o = *opts;
  SolveSpec sp;
  sp.solver = solver;
  sp.rel_tol = rel_tol;
  sp.maxit = max_iters;
  sp.restart = o.restart > 0 ? o.restart : 30;
  if (sp.restart > kMaxRestart) return fail(GKO_INVALID_ARG, "GMRES restart length is limited to 128");
  sp.check_true = 1;
  sp.check_every = o.check_every;
  if (o.preconditioner != GKO_PRECOND_NONE && o.preconditioner != GKO_PRECOND_JACOBI &&
      o.preconditioner != GKO_PRECOND_BLOCK_JACOBI)
    return fail(GKO_INVALID_ARG, "unknown preconditioner");
  const bool jacobi = o.preconditioner == GKO_PRECOND_JACOBI;
  const bool bjac = o.preconditioner == GKO_PRECOND_BLOCK_JACOBI;
  if ((jacobi || bjac) && solver == 2) return fail(GKO_NOT_SUPPORTED, "GMRES takes no preconditioner");
  const int bsize = o.block_size > 0 ? o.block_size : 8;
  if (bjac) {
    if (bsize > kBlockJacobiMax) return fail(GKO_INVALID_ARG, "block-Jacobi block size must lie in 1..32");
    if (A->fmt != GKO_CSR) return fail(GKO_NOT_SUPPORTED, "the block-Jacobi setup reads a CSR matrix");
  }
  double nb = 0.0;
  GKO_TRY(norm2_host(b, n, &nb, s));
  Scratch pc_mem;  // Jacobi inverse diagonal: FP64, and its FP32 rounding for inner solves
  double* d64 = nullptr;
  if (jacobi) {
    GKO_TRY(pc_mem.get(sizeof(double) * n + sizeof(float) * n + 512, s));
    d64 = pc_mem.as<double>();
    GKO_TRY(jacobi_inverse(A, d64, s));
    sp.minv = d64;
  }
  Scratch bj_mem;  // block-Jacobi: n x bs inverse-block rows (FP64), and their FP32 rounding
  const size_t bj_count = bjac ? (size_t)n * bsize : 0;
  const size_t bj32_off = ((sizeof(double) * bj_count + 255) / 256) * 256;
  if (bjac) {
    const bool mixed = o.precision != GKO_PRECISION_F64;
    GKO_TRY(bj_mem.get(bj32_off + (mixed ? sizeof(float) * bj_count : 0) + 512, s));
    GKO_TRY(block_jacobi_inverse(A, bsize, bj_mem.as<double>(), nullptr, s));
    sp.bj = bj_mem.as<double>();
    sp.bs = bsize;
  }

  if (o.precision == GKO_PRECISION_F64) {
    SolveOut so{};
    GKO_TRY(krylov_core<double>(A, b, x, false, sp, s, &so));
    res->iterations = so.iterations;
    res->outer_iterations = so.cycles;
    GKO_TRY(true_rel_residual(A, b, x, nb, &res->rel_residual, s));
    res->status = map_status(so.status);
    return res->status;
  }
  if (o.precision != GKO_PRECISION_MIXED_F32 && o.precision != GKO_PRECISION_MIXED_BF16)
    return fail(GKO_INVALID_ARG, "unknown precision");
  if (o.refinement != GKO_REFINE_AUTO && o.refinement != GKO_REFINE_RESTART && o.refinement != GKO_REFINE_RELIABLE)
    return fail(GKO_INVALID_ARG, "unknown refinement");
  if (o.refinement == GKO_REFINE_RELIABLE && solver == 2)
    return fail(GKO_NOT_SUPPORTED, "GMRES refines by restarting (reliable updates are for CG and BiCGSTAB)");
  if (!(o.reliable_delta >= 0.0 && o.reliable_delta < 1.0))
    return fail(GKO_INVALID_ARG, "reliable_delta must lie in [0, 1)");
  // AUTO: reliable updates for BiCGSTAB, and for CG where the single-launch
  // small-system CG (which refines by restarting) does not apply
  const bool reliable = o.refinement == GKO_REFINE_RELIABLE ||
                        (o.refinement == GKO_REFINE_AUTO && (solver == 1 || (solver == 0 && n > kSmallRows)));
  gko_matrix A32 = nullptr;
  GKO_TRY(lowp_copy(A, o.precision == GKO_PRECISION_MIXED_F32 ? GKO_F32 : GKO_BF16, s, &A32));
  // mixed-precision iterative refinement: FP64 residual, FP32-stored inner solve
  SolveSpec in = sp;
  if (jacobi) {
    float* d32 = pc_mem.as<float>(((sizeof(double) * (size_t)n + 255) / 256) * 256);
    GKO_TRY(narrow_to_f32(d64, d32, n, s));
    in.minv = d32;
  }
  if (bjac) {  // the inner recurrences apply the FP32-rounded inverse blocks
    float* b32 = bj_mem.as<float>(bj32_off);
    GKO_TRY(narrow_to_f32(bj_mem.as<double>(), b32, (int64_t)bj_count, s));
    in.bj = b32;
  }
  in.rel_tol = o.inner_tol > 0 ? o.inner_tol : 1e-5;
  // GMRES: at most 4 restart cycles per refinement step by default.  An
  // inner FP32 GMRES left to restart on its own FP32 residual until the
  // inner tolerance needed a third more iterations on 128^3 convection-
  // diffusion (863 vs 645 in FP64); with 1, 2 or 4 cycles per step it takes
  // 653 (227 ms against 273 ms in FP64 whichever), and 4 needs the fewest
  // FP64 residuals.  Up to max_iters inner iterations in all.
  const bool gmres = solver == 2;
  const int gmres_inner = 4 * sp.restart;
  in.maxit = o.inner_maxit > 0 ? o.inner_maxit : (gmres ? gmres_inner : max_iters);
  in.check_true = 0;
  const int max_outer =
      o.max_outer > 0 ? o.max_outer : (gmres ? std::max(30, (max_iters + gmres_inner - 1) / gmres_inner) : 30);
  Scratch mem;
  const size_t sb = spmv_scratch_bytes(A);
  GKO_TRY(mem.get(sizeof(double) * n + sizeof(float) * n + sb + 2048, s));
  Carve cv{static_cast<char*>(mem.data())};
  double* r = cv.take<double>(n);
  float* d = cv.take<float>(n);
  void* ss = sb ? cv.take<char>(sb) : nullptr;
  const int vg = vec_grid(n);
  int total_inner = 0, outer = 0;
  bool converged = nb == 0.0;
  if (nb == 0.0) zero_kernel<double><<<vg, 256, 0, s>>>(n, x);
  if (reliable && !converged) {
    // one run of the FP32 recurrences from fl32(b - A x); updates fold d into
    // x and replace the recurrence residual until ||b - A x|| <= rel_tol ||b||
    GKO_TRY(spmv_run(A, x, r, 1.0, 0.0, s, ss, nullptr, nullptr));
    residual64_kernel<<<vg, 256, 0, s>>>(n, b, r);
    GKO_TRY_CUDA(cudaGetLastError());
    double nr = 0.0;
    GKO_TRY(norm2_host(r, n, &nr, s));
    if (nr <= rel_tol * nb) {
      converged = true;
    } else {
      // r is read once to start the recurrences, then serves as the FP64
      // product A x of every update
      RelSpec rl{A, b, x, r, ss, o.reliable_delta > 0.0 ? o.reliable_delta : 0.1};
      SolveSpec step = in;
      step.rel = &rl;
      step.check_true = 1;
      step.maxit = max_iters;
      step.rel_tol = rel_tol * nb / nr;
      SolveOut so{};
      GKO_TRY(krylov_core<float>(A32, r, d, true, step, s, &so));
      res->iterations = so.iterations;
      res->outer_iterations = so.cycles;
      GKO_TRY(true_rel_residual(A, b, x, nb, &res->rel_residual, s));
      res->status = map_status(so.status);
      return res->status;
    }
  }
  while (!converged) {
    GKO_TRY(spmv_run(A, x, r, 1.0, 0.0, s, ss, nullptr, nullptr));
    residual64_kernel<<<vg, 256, 0, s>>>(n, b, r);
    GKO_TRY_CUDA(cudaGetLastError());
    double nr = 0.0;
    GKO_TRY(norm2_host(r, n, &nr, s));
    if (nr <= rel_tol * nb) {
      converged = true;
      break;
    }
    if (outer >= max_outer) break;
    // ask the inner solve only for the reduction still needed (with a factor
    // 2 margin), never tighter than inner_tol
    SolveSpec step = in;
    step.rel_tol = std::max(in.rel_tol, std::min(0.5, 0.5 * rel_tol * nb / nr));
    SolveOut so{};
    GKO_TRY(krylov_core<float>(A32, r, d, true, step, s, &so));
    total_inner += so.iterations;
    outer += 1;
    add_f32_kernel<<<vg, 256, 0, s>>>(n, x, d);
    GKO_TRY_CUDA(cudaGetLastError());
  }
  res->iterations = total_inner;
  res->outer_iterations = outer;
  GKO_TRY(true_rel_residual(A, b, x, nb, &res->rel_residual, s));
  res->status = converged ? GKO_OK : GKO_NOT_CONVERGED;
  return res->status;
}

}  // namespace gko

extern "C" {

int gko_solve_cg(gko_matrix A, const double* b, double* x, double rel_tol, int32_t max_iters,
                 const gko_solve_opts* opts, gko_solve_result* res, void* stream) {
  return gko::solve_entry(0, A, b, x, rel_tol, max_iters, opts, res, stream);
}

int gko_solve_bicgstab(gko_matrix A, const double* b, double* x, double rel_tol, int32_t max_iters,
                       const gko_solve_opts* opts, gko_solve_result* res, void* stream) {
  return gko::solve_entry(1, A, b, x, rel_tol, max_iters, opts, res, stream);
}

int gko_solve_gmres(gko_matrix A, const double* b, double* x, double rel_tol, int32_t max_iters,
                    const gko_solve_opts* opts, gko_solve_result* res, void* stream) {
  return gko::solve_entry(2, A, b, x, rel_tol, max_iters, opts, res, stream);
}

}  // extern "C"
