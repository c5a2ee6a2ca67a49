// SpMV dispatch over value types and the gko_spmv entry point.
#include <algorithm>
#include <utility>
#include <vector>

#include "spmv.cuh"

namespace gko {

size_t spmv_scratch_bytes(const gko_matrix_s* A) {
  const size_t at = A->dtype == GKO_F64 ? 8 : 4;
  switch (A->fmt) {
    case GKO_CSR:
      if (A->plan.kind == 2) return at * 2 * (size_t)((A->n_rows + A->nnz + 2047) / 2048 + 1);
      if (A->plan.kind == 3) return at * 2 * (size_t)((A->nnz + kCooTile - 1) / kCooTile + 1);
      return at * (size_t)A->plan.n_chunks;
    case GKO_ELL:
    case GKO_SELLP:
      return 0;
    case GKO_COO:
      if (A->plan.kind == 1) return 0;
      return at * 2 * (size_t)((A->coo_nnz + kCooTile - 1) / kCooTile);
    case GKO_HYBRID:
      return at * 2 * (size_t)((A->coo_nnz + kCooTile - 1) / kCooTile);
  }
  return 0;
}

bool spmv_fuses_dot(const gko_matrix_s* A) {
  return (A->fmt == GKO_CSR && A->plan.kind != 2 && A->plan.kind != 3) || A->fmt == GKO_ELL || A->fmt == GKO_SELLP ||
         (A->fmt == GKO_COO && A->plan.kind == 1 && A->coo_nnz > 0);
}

int spmv_run(const gko_matrix_s* A, const void* x, void* y, double alpha, double beta, cudaStream_t s, void* scratch,
             const DotSpec* dot, const int* gate) {
  switch (A->dtype) {
    case GKO_F64:
      return spmv_run_f64(A, static_cast<const double*>(x), static_cast<double*>(y), alpha, beta, s, scratch, dot, gate);
    case GKO_F32:
      return spmv_run_f32(A, static_cast<const float*>(x), static_cast<float*>(y), alpha, beta, s, scratch, dot, gate);
    case GKO_BF16:
      return spmv_run_bf16(A, static_cast<const float*>(x), static_cast<float*>(y), alpha, beta, s, scratch, dot, gate);
  }
  return fail(GKO_INVALID_ARG, "bad dtype");
}

}  // namespace gko

using namespace gko;

extern "C" int gko_spmv(const double* alpha, gko_matrix A, const void* x, const double* beta, void* y,
                        gko_dtype vec_dtype, void* stream) {
  if (!A || !alpha || !beta) return fail(GKO_INVALID_ARG, "null matrix or scalar");
  if (A->n_rows > 0 && !y) return fail(GKO_INVALID_ARG, "null y");
  if (A->n_cols > 0 && A->nnz > 0 && !x) return fail(GKO_INVALID_ARG, "null x");
  const gko_dtype need = A->dtype == GKO_F64 ? GKO_F64 : GKO_F32;
  if (vec_dtype != need)
    return fail(GKO_INVALID_ARG, "vector dtype must be F64 for F64 matrices and F32 for F32/BF16 matrices");
  if (A->n_rows == 0) return GKO_OK;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scratch;
  const size_t sb = spmv_scratch_bytes(A);
  if (sb) GKO_TRY(scratch.get(sb, s));
  return spmv_run(A, x, y, *alpha, *beta, s, scratch.data(), nullptr);
}

// SpMV on host vectors: stream-ordered copies around gko_spmv (see gko.h).
extern "C" int gko_spmv_host(const double* alpha, gko_matrix A, const void* x_host, const double* beta,
                             void* y_host, gko_dtype vec_dtype, void* x_dev, void* y_dev, void* stream) {
  if (!A || !alpha || !beta) return fail(GKO_INVALID_ARG, "null matrix or scalar");
  if (A->n_rows > 0 && (!y_host || !y_dev)) return fail(GKO_INVALID_ARG, "null y");
  if (A->n_cols > 0 && (!x_host || !x_dev)) return fail(GKO_INVALID_ARG, "null x");
  const size_t es = vec_dtype == GKO_F64 ? sizeof(double) : sizeof(float);
  cudaStream_t s = (cudaStream_t)stream;
  if (A->n_cols > 0)
    GKO_TRY_CUDA(cudaMemcpyAsync(x_dev, x_host, es * (size_t)A->n_cols, cudaMemcpyHostToDevice, s));
  if (A->n_rows > 0 && *beta != 0.0)
    GKO_TRY_CUDA(cudaMemcpyAsync(y_dev, y_host, es * (size_t)A->n_rows, cudaMemcpyHostToDevice, s));
  GKO_TRY(gko_spmv(alpha, A, x_dev, beta, y_dev, vec_dtype, stream));
  if (A->n_rows > 0)
    GKO_TRY_CUDA(cudaMemcpyAsync(y_host, y_dev, es * (size_t)A->n_rows, cudaMemcpyDeviceToHost, s));
  return GKO_OK;
}

// Autotuner of the SpMV plan (see gko.h): times each candidate plan on the
// caller's vectors with L2 flushed before every timed SpMV, keeps the best.
extern "C" int gko_matrix_tune(gko_matrix m, const void* x, void* y, int32_t reps, int32_t keep_kernel,
                               int32_t* kernel, int32_t* S, int32_t* R, int32_t* cap, float* best_ms, void* stream) {
  if (!m || reps < 1 || reps > 100) return fail(GKO_INVALID_ARG, "bad tune arguments (reps 1..100)");
  if (m->fmt != GKO_CSR && m->fmt != GKO_COO) return fail(GKO_NOT_SUPPORTED, "tuning covers CSR and COO plans");
  if (m->n_rows > 0 && (!x || !y)) return fail(GKO_INVALID_ARG, "null x or y");
  cudaStream_t s = (cudaStream_t)stream;
  struct Cand {
    int32_t k, S, R, cap;
  };
  std::vector<Cand> cands;
  const Cand start{m->plan.kind, m->plan.S, m->plan.R, m->plan.cap};
  // keep_kernel: only the parameters of the handle's current kernel (the
  // row-block plans; merge path and segmented reduction have none)
  if (!keep_kernel || start.k == 1)
    for (int32_t ss : {1, 2, 4, 8})
      for (int32_t rr : {1, 2, 4})
        for (int32_t cc : {512, 1024, 2048}) cands.push_back({1, ss, rr, cc});
  if (!keep_kernel) {
    if (m->fmt == GKO_CSR) {
      cands.push_back({2, 1, 1, 1024});  // merge path
      cands.push_back({3, 1, 1, 1024});  // nonzero split
      for (int32_t ss : {4, 8, 16, 32}) cands.push_back({0, ss, 2, 1024});
    } else {
      cands.push_back({0, 1, 1, 1024});  // segmented reduction
    }
  }
  if (cands.empty()) cands.push_back(start);
  if (m->n_rows == 0) {
    if (kernel) *kernel = start.k;
    if (S) *S = start.S;
    if (R) *R = start.R;
    if (cap) *cap = start.cap;
    if (best_ms) *best_ms = 0.f;
    return GKO_OK;
  }
  const size_t flush_bytes = 256u << 20;  // larger than the 129 MB L2
  Scratch flush;
  GKO_TRY(flush.get(flush_bytes, s));
  struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  GKO_TRY_CUDA(cudaEventCreate(&ev.a));
  GKO_TRY_CUDA(cudaEventCreate(&ev.b));
  const double one = 1.0, zero = 0.0;
  const gko_dtype vdt = m->dtype == GKO_F64 ? GKO_F64 : GKO_F32;
  // Fastest of `n` L2-flushed runs of candidate c (1e30 if it does not apply).
  auto time_plan = [&](const Cand& c, int n, float* out) -> int {
    *out = 1e30f;
    if (gko_matrix_set_plan(m, c.k, c.S, c.R, c.cap, stream) != GKO_OK) return GKO_OK;  // not applicable here
    GKO_TRY(gko_spmv(&one, m, x, &zero, y, vdt, stream));  // first use of this configuration
    for (int r = 0; r < n; ++r) {
      GKO_TRY_CUDA(cudaMemsetAsync(flush.data(), r & 0xff, flush_bytes, s));
      GKO_TRY_CUDA(cudaEventRecord(ev.a, s));
      GKO_TRY(gko_spmv(&one, m, x, &zero, y, vdt, stream));
      GKO_TRY_CUDA(cudaEventRecord(ev.b, s));
      GKO_TRY_CUDA(cudaEventSynchronize(ev.b));
      float ms = 0.f;
      GKO_TRY_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
      *out = std::min(*out, ms);
    }
    return GKO_OK;
  };
  // First pass: every candidate, `reps` runs.  Second pass: the three fastest
  // again with 3*reps runs, so a single lucky run cannot pick the plan.
  std::vector<std::pair<float, size_t>> t1;
  for (size_t i = 0; i < cands.size(); ++i) {
    float t = 1e30f;
    GKO_TRY(time_plan(cands[i], reps, &t));
    if (t < 1e30f) t1.push_back({t, i});
  }
  std::sort(t1.begin(), t1.end());
  float best = 1e30f;
  Cand best_c = start;
  for (size_t j = 0; j < t1.size() && j < 3; ++j) {
    float t = 1e30f;
    GKO_TRY(time_plan(cands[t1[j].second], 3 * reps, &t));
    if (t < best) {
      best = t;
      best_c = cands[t1[j].second];
    }
  }
  GKO_TRY(gko_matrix_set_plan(m, best_c.k, best_c.S, best_c.R, best_c.cap, stream));
  if (kernel) *kernel = best_c.k;
  if (S) *S = best_c.S;
  if (R) *R = best_c.R;
  if (cap) *cap = best_c.cap;
  if (best_ms) *best_ms = best;
  return GKO_OK;
}

