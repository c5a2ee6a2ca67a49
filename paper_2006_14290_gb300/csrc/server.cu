// Serving runtime (host C++): a request loop over resident matrices with
// continuous batching.  Requests (matrix id, solver, right-hand side,
// tolerance) are queued as they arrive; `slots` worker threads, each with
// its own CUDA stream, take the oldest request as soon as a slot is free and
// its memory estimate fits the HBM budget, so new work starts while other
// solves are still on the GPU and their kernels overlap on the device.
// Every solve uses the library's deterministic kernels, so a result does not
// depend on what else is running.  Latency is measured from submission to
// the moment the solution is back on the host.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  int32_t matrix = 0;
  gko_matrix A = nullptr;  // the resident matrix and its size, copied at submission under the lock
  int64_t n = 0;
  int32_t solver = 0;
  double tol = 1e-8;
  int32_t maxit = 1000;
  gko_solve_opts opts{};
  bool has_opts = false;
  std::vector<double> b, x;
  int64_t bytes = 0;
  Clock::time_point t_submit, t_start, t_done;
  gko_solve_result res{};
  int code = GKO_OK;
  bool done = false;
};

struct Resident {
  gko_matrix A = nullptr;
  int64_t n = 0;
  int64_t bytes = 0;
};

}  // namespace

struct gko_server_s {
  int device = 0;
  int32_t slots = 1;
  int64_t budget = 0;  // bytes for matrices + in-flight workspaces (0: unlimited)
  int64_t resident_bytes = 0;
  int64_t inflight_bytes = 0;
  std::vector<Resident> matrices;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<int64_t, std::shared_ptr<Request>> requests;
  std::vector<double> latencies_ms;
  int64_t next_id = 1;
  int64_t completed = 0;
  int32_t active = 0, peak_active = 0;
  bool stop = false;
  Clock::time_point t_first, t_last;
  bool any = false;
  std::vector<std::thread> workers;
};

namespace {

// Device bytes one request holds while it runs: b and x, the solver's
// vectors (CG 4, BiCGSTAB 8, GMRES restart+3 of length n; with a
// preconditioner one more for CG's z and two for BiCGSTAB's preconditioned
// directions), for mixed precision the FP32 inner vectors, and the
// preconditioner itself (Jacobi: the inverse diagonal and its FP32
// rounding; block-Jacobi: block_size inverse-block entries per row, FP64
// and, for mixed precision, FP32).
int64_t request_bytes(const Request& r, int64_t n) {
  const int restart = r.has_opts && r.opts.restart > 0 ? r.opts.restart : 30;
  const int pc = r.has_opts ? r.opts.preconditioner : GKO_PRECOND_NONE;
  int vecs = r.solver == 0 ? 4 : r.solver == 1 ? 8 : restart + 3;
  if (pc != GKO_PRECOND_NONE) vecs += r.solver == 0 ? 1 : 2;
  const bool mixed = r.has_opts && r.opts.precision != GKO_PRECISION_F64;
  int64_t per = mixed ? (int64_t)(vecs * 4 + 2 * 8 + 8) : (int64_t)(vecs * 8);
  if (pc == GKO_PRECOND_JACOBI) per += 8 + 4;
  if (pc == GKO_PRECOND_BLOCK_JACOBI) {
    const int bs = r.opts.block_size > 0 ? r.opts.block_size : 8;
    per += (int64_t)bs * (mixed ? 12 : 8);
  }
  return (per + 16) * n + (4 << 20);
}

void worker_loop(gko_server S) {
  cudaSetDevice(S->device);
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return;
  double* pin = nullptr;
  size_t pin_n = 0;
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] {
        if (S->stop) return true;
        if (S->queue.empty()) return false;
        const int64_t need = S->queue.front()->bytes;
        return S->budget <= 0 || S->resident_bytes + S->inflight_bytes + need <= S->budget;
      });
      if (S->stop) break;
      r = S->queue.front();
      S->queue.pop_front();
      S->inflight_bytes += r->bytes;
      S->active += 1;
      S->peak_active = std::max(S->peak_active, S->active);
    }
    r->t_start = Clock::now();
    const int64_t n = r->n;
    int code = GKO_OK;
    gko::Scratch dev;
    if ((size_t)n > pin_n) {
      if (pin) cudaFreeHost(pin);
      pin = nullptr;
      pin_n = 0;
      if (cudaMallocHost((void**)&pin, sizeof(double) * (size_t)n) == cudaSuccess) pin_n = (size_t)n;
    }
    code = dev.get(sizeof(double) * 2 * (size_t)n + 512, s);
    if (code == GKO_OK && pin) {
      double* db = dev.as<double>();
      double* dx = dev.as<double>(((sizeof(double) * (size_t)n + 255) / 256) * 256);
      std::copy(r->b.begin(), r->b.end(), pin);
      const gko_solve_opts* o = r->has_opts ? &r->opts : nullptr;
      if (cudaMemcpyAsync(db, pin, sizeof(double) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
          cudaMemsetAsync(dx, 0, sizeof(double) * n, s) != cudaSuccess) {
        cudaGetLastError();
        code = GKO_CUDA_ERROR;
      } else if (r->solver == 0) code = gko_solve_cg(r->A, db, dx, r->tol, r->maxit, o, &r->res, s);
      else if (r->solver == 1) code = gko_solve_bicgstab(r->A, db, dx, r->tol, r->maxit, o, &r->res, s);
      else code = gko_solve_gmres(r->A, db, dx, r->tol, r->maxit, o, &r->res, s);
      if (code == GKO_OK || code == GKO_NOT_CONVERGED || code == GKO_BREAKDOWN) {
        if (cudaMemcpyAsync(pin, dx, sizeof(double) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
          code = GKO_CUDA_ERROR;
        else
          r->x.assign(pin, pin + n);
      }
    } else if (code == GKO_OK) {
      code = GKO_OUT_OF_MEMORY;
    }
    cudaStreamSynchronize(s);
    r->t_done = Clock::now();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      r->code = code;
      r->done = true;
      S->inflight_bytes -= r->bytes;
      S->active -= 1;
      S->completed += 1;
      S->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
      S->t_last = r->t_done;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  if (pin) cudaFreeHost(pin);
  cudaStreamDestroy(s);
}

}  // namespace

using namespace gko;

extern "C" {

int gko_server_create(int32_t slots, int64_t budget_bytes, gko_server* out) {
  if (!out || slots < 1 || slots > 64 || budget_bytes < 0) return fail(GKO_INVALID_ARG, "bad server arguments");
  std::unique_ptr<gko_server_s> S(new gko_server_s());
  GKO_TRY_CUDA(cudaGetDevice(&S->device));
  S->slots = slots;
  S->budget = budget_bytes;
  for (int i = 0; i < slots; ++i) S->workers.emplace_back(worker_loop, S.get());
  *out = S.release();
  return GKO_OK;
}

int gko_server_add_matrix(gko_server S, gko_matrix A, int32_t* matrix_id) {
  if (!S || !A || !matrix_id) return fail(GKO_INVALID_ARG, "null argument");
  if (A->n_rows != A->n_cols || A->dtype != GKO_F64) return fail(GKO_INVALID_ARG, "server matrices are square F64");
  int64_t bytes = 0;
  GKO_TRY(gko_matrix_info(A, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, &bytes));
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->budget > 0 && S->resident_bytes + bytes > S->budget)
    return fail(GKO_BUDGET_EXCEEDED, "resident matrices exceed the server budget");
  S->matrices.push_back(Resident{A, A->n_rows, bytes});
  S->resident_bytes += bytes;
  *matrix_id = (int32_t)S->matrices.size() - 1;
  return GKO_OK;
}

int gko_server_submit(gko_server S, int32_t matrix_id, int32_t solver, const double* b, double rel_tol,
                      int32_t max_iters, const gko_solve_opts* opts, int64_t* request_id) {
  if (!S || !b || !request_id) return fail(GKO_INVALID_ARG, "null argument");
  auto r = std::make_shared<Request>();
  r->t_submit = Clock::now();
  if (solver < 0 || solver > 2 || !(rel_tol >= 0.0) || max_iters < 0) return fail(GKO_INVALID_ARG, "bad request");
  {
    // the request keeps its own copy of the handle and size: add_matrix may
    // grow the matrix table while solves run
    std::lock_guard<std::mutex> lk(S->mu);
    if (matrix_id < 0 || matrix_id >= (int32_t)S->matrices.size())
      return fail(GKO_INVALID_ARG, "unknown matrix id");
    r->A = S->matrices[matrix_id].A;
    r->n = S->matrices[matrix_id].n;
  }
  const int64_t n = r->n;
  r->matrix = matrix_id;
  r->solver = solver;
  r->tol = rel_tol;
  r->maxit = max_iters;
  if (opts) {
    r->opts = *opts;
    r->has_opts = true;
  }
  r->b.assign(b, b + n);
  r->bytes = request_bytes(*r, n);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->budget > 0 && S->resident_bytes + r->bytes > S->budget)
      return fail(GKO_BUDGET_EXCEEDED, "request needs more memory than the server budget leaves");
    r->id = S->next_id++;
    if (!S->any) {
      S->t_first = r->t_submit;
      S->any = true;
    }
    S->requests[r->id] = r;
    S->queue.push_back(r);
    *request_id = r->id;
  }
  S->cv_work.notify_one();
  return GKO_OK;
}

// Non-blocking (wait == 0) or blocking wait for a request.  On completion
// copies the solution (x, n doubles, optional) and the result, reports the
// latency in milliseconds, and forgets the request.  *done = 0 while running.
int gko_server_result(gko_server S, int64_t request_id, int wait, int32_t* done, gko_solve_result* res, double* x,
                      double* latency_ms) {
  if (!S || !done) return fail(GKO_INVALID_ARG, "null argument");
  std::shared_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->requests.find(request_id);
    if (it == S->requests.end()) return fail(GKO_INVALID_ARG, "unknown request id");
    r = it->second;
    if (wait) S->cv_done.wait(lk, [&] { return r->done; });
    *done = r->done ? 1 : 0;
    if (!r->done) return GKO_OK;
    S->requests.erase(it);
  }
  if (res) *res = r->res;
  if (x && !r->x.empty()) std::copy(r->x.begin(), r->x.end(), x);
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  return r->code;
}

int gko_server_stats(gko_server S, int64_t* completed, double* p50_ms, double* p99_ms, double* solves_per_s,
                     int32_t* peak_active) {
  if (!S) return fail(GKO_INVALID_ARG, "null server");
  std::vector<double> lat;
  double span = 0.0;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    lat = S->latencies_ms;
    if (completed) *completed = S->completed;
    if (peak_active) *peak_active = S->peak_active;
    if (S->any && S->completed) span = std::chrono::duration<double>(S->t_last - S->t_first).count();
  }
  std::sort(lat.begin(), lat.end());
  auto pct = [&](double q) -> double {
    if (lat.empty()) return 0.0;
    const size_t k = std::min(lat.size() - 1, (size_t)(q * (double)(lat.size() - 1) + 0.5));
    return lat[k];
  };
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  if (solves_per_s) *solves_per_s = span > 0 ? (double)lat.size() / span : 0.0;
  return GKO_OK;
}

int gko_server_destroy(gko_server S) {
  if (!S) return GKO_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  delete S;
  return GKO_OK;
}

}  // extern "C"
