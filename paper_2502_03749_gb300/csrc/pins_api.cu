// C ABI of the library (include/pins.h): handles, blocking and batched solves,
// and the serving path (pins_submit / pins_poll / pins_wait).
//
// Serving design: requests are deep-copied into host memory at submit and
// queued.  A fixed pool of worker threads, each owning one CUDA stream and one
// Solver (device workspace arena), takes requests in arrival order when (a) the
// worker is idle and (b) every arena the pool holds -- those of running
// requests and those idle workers keep for reuse -- fits the device budget with
// the new request's workspace.  Idle workers' arenas are released when that is
// what makes a request fit.  Running requests overlap on the device through
// their streams; each keeps its potentials, CSR pattern and CG vectors resident
// in its own arena for its whole solve.  All kernels reduce in a fixed order, so
// a result does not depend on what else runs.
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>
#include "pins_solver.h"

using pins::Solver;

namespace {

struct OwnedProblem {
  pins_problem p{};
  std::vector<double> a, b, x, y, C64;
  std::vector<float> C32;
  std::vector<double> F, G;   // results
};

struct Job {
  uint64_t ticket = 0;
  OwnedProblem prob;
  pins_result res{};
  pins_status status = PINS_ERR_PENDING;
  bool done = false;
  size_t need = 0;
  std::string error;
};

}  // namespace

struct pins_handle {
  pins_config cfg{};
  int device = 0;
  int sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  float2* exp_table = nullptr;
  std::unique_ptr<Solver> solver;
  std::string last_error;
  std::mutex err_mu;
  // serving
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Job>> queue;
  std::map<uint64_t, std::shared_ptr<Job>> jobs;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> worker_streams;
  std::vector<std::unique_ptr<Solver>> worker_solvers;
  std::vector<size_t> held;      // per worker: arena bytes held (reserved while running)
  std::vector<char> busy;        // per worker: running a request
  pins::FaultHooks hooks;        // host-side fault injection (tests)
  size_t budget = 0;
  int running = 0;
  bool stopping = false;
  uint64_t next_ticket = 1;
};

static void set_error(pins_handle* h, const std::string& e) {
  std::lock_guard<std::mutex> g(h->err_mu);
  h->last_error = e;
}

extern "C" void pins_config_default(pins_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->eta = 1e-2;
  c->tol_marg = 1e-9;
  c->tol_gap = 0.0;
  c->cg_rtol = 1e-6;
  c->armijo_beta = 0.5;
  c->armijo_c1 = 1e-4;
  c->sparsify_gamma = 1.0;
  c->T1 = 100;
  c->T2 = 50;
  c->K = 250;
  c->max_cg = 1000;
  c->max_backtrack = 30;
  c->sinkhorn_check_every = 10;
  c->gap_every = 1;
  c->prec = PINS_PREC_FP64;
  c->device = 0;
  c->cuda_stream = nullptr;
  c->max_inflight = 4;
  c->queue_capacity = 4096;
  c->device_mem_budget = 0;
  c->sparsify_one_pass = 1;
}

static bool config_ok(const pins_config& c, std::string& why) {
  if (!(c.eta > 0.0) || !std::isfinite(c.eta)) { why = "eta must be > 0"; return false; }
  if (!(c.tol_marg >= 0.0) || !(c.tol_gap >= 0.0) || !(c.cg_rtol > 0.0)) { why = "tolerances must be >= 0"; return false; }
  if (!(c.armijo_beta > 0.0 && c.armijo_beta < 1.0)) { why = "armijo_beta must be in (0,1)"; return false; }
  if (!(c.armijo_c1 > 0.0 && c.armijo_c1 < 1.0)) { why = "armijo_c1 must be in (0,1)"; return false; }
  if (!(c.sparsify_gamma > 0.0)) { why = "sparsify_gamma must be > 0"; return false; }
  if (c.T1 < 0 || c.T2 < 0 || c.K < 1 || c.max_cg < 1 || c.max_backtrack < 0) { why = "iteration caps out of range"; return false; }
  if (c.T1 > 1000000) { why = "T1 too large"; return false; }
  if (c.prec != PINS_PREC_FP64 && c.prec != PINS_PREC_MIXED) { why = "unknown precision"; return false; }
  if (c.max_inflight < 1 || c.max_inflight > 64 || c.queue_capacity < 1) { why = "serving limits out of range"; return false; }
  return true;
}

static std::vector<float2> make_exp_table() {
  std::vector<float2> t(PINS_EXP_TABLE);
  for (int q = 0; q < PINS_EXP_TABLE; ++q) {
    double v = std::exp2((double)q / PINS_EXP_TABLE);
    float hi = (float)v;
    t[q] = make_float2(hi, (float)(v - (double)hi));
  }
  return t;
}

extern "C" pins_status pins_create(const pins_config* cfg, pins_handle** out) {
  if (!cfg || !out) return PINS_ERR_INVALID_ARG;
  *out = nullptr;
  std::string why;
  if (!config_ok(*cfg, why)) return PINS_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) { cudaGetLastError(); return PINS_ERR_CUDA; }
  if (cfg->device < 0 || cfg->device >= ndev) return PINS_ERR_INVALID_ARG;
  if (cudaSetDevice(cfg->device) != cudaSuccess) { cudaGetLastError(); return PINS_ERR_CUDA; }
  auto* h = new pins_handle();
  h->cfg = *cfg;
  h->device = cfg->device;
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  if (cfg->cuda_stream) h->stream = (cudaStream_t)cfg->cuda_stream;
  else {
    // a blocking stream: ordered after work the caller queued on the legacy
    // default stream (e.g. the fills that produced device inputs)
    if (cudaStreamCreate(&h->stream) != cudaSuccess) { delete h; return PINS_ERR_CUDA; }
    h->own_stream = true;
  }
  std::vector<float2> tab = make_exp_table();
  if (cudaMalloc(&h->exp_table, sizeof(float2) * tab.size()) != cudaSuccess) {
    cudaGetLastError();
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return PINS_ERR_OOM;
  }
  cudaMemcpy(h->exp_table, tab.data(), sizeof(float2) * tab.size(), cudaMemcpyHostToDevice);
  h->solver.reset(new Solver(h->device, h->sms, h->exp_table));
  h->solver->set_stream(h->stream);
  h->solver->set_hooks(&h->hooks);
  h->solver->set_profile(cfg->profile != 0);
  size_t freeb = 0, totalb = 0;
  cudaMemGetInfo(&freeb, &totalb);
  h->budget = cfg->device_mem_budget ? cfg->device_mem_budget : (size_t)(0.8 * (double)freeb);
  if (cudaGetLastError() != cudaSuccess) { pins_destroy(h); return PINS_ERR_CUDA; }
  *out = h;
  return PINS_OK;
}

extern "C" void pins_destroy(pins_handle* h) {
  if (!h) return;
  {
    std::lock_guard<std::mutex> g(h->mu);
    h->stopping = true;
  }
  h->cv_work.notify_all();
  for (auto& t : h->workers) t.join();
  cudaSetDevice(h->device);
  h->worker_solvers.clear();
  for (auto s : h->worker_streams) cudaStreamDestroy(s);
  h->solver.reset();
  if (h->exp_table) cudaFree(h->exp_table);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

extern "C" int pins_profile_classes(void) { return Solver::PC_COUNT; }

extern "C" const char* pins_profile_name(int k) { return Solver::prof_name(k); }

extern "C" pins_status pins_profile_read(pins_handle* h, double* ms, long long* launches, int n,
                                         int reset) {
  if (!h || n < 0) return PINS_ERR_INVALID_ARG;
  h->solver->prof_read(ms, launches, n, reset != 0);
  return PINS_OK;
}

extern "C" const char* pins_last_error(pins_handle* h) {
  if (!h) return "null handle";
  std::lock_guard<std::mutex> g(h->err_mu);
  return h->last_error.c_str();
}

extern "C" pins_status pins_solve(pins_handle* h, const pins_problem* p, pins_result* r) {
  if (!h || !p || !r) return PINS_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  pins_status s = h->solver->solve(h->cfg, *p, *r);
  if (s != PINS_OK) set_error(h, h->solver->error().empty() ? "not converged" : h->solver->error());
  return s;
}

// ------------------------------------------------------------------------- //
// serving
// ------------------------------------------------------------------------- //
static size_t job_need(const pins_config& cfg, const pins_problem& p) {
  return pins::solve_workspace_bytes(cfg, p);
}

// Admission of the queue's head by worker idx (h->mu held).  The pool holds at
// most budget bytes of arenas: the other workers' arenas (running, or kept by
// idle workers for reuse) plus what this worker holds for the request -- its
// own arena if it is at least the need and at most twice it, else a fresh one
// of the need.  Idle workers' arenas are released while the pool would exceed
// the budget.  A request always runs when nothing else is running (submit has
// rejected any request whose need alone exceeds the budget).  The handle's own
// blocking solver (pins_solve) is not part of this pool.
static bool admit(pins_handle* h, int idx, size_t need) {
  const size_t mine = h->held[idx];
  size_t others = 0;
  for (size_t k = 0; k < h->held.size(); ++k)
    if ((int)k != idx) others += h->held[k];
  bool keep = mine >= need && mine <= 2 * need;
  size_t after = keep ? mine : need;
  for (size_t k = 0; k < h->held.size() && others + after > h->budget; ++k) {
    if ((int)k == idx || h->busy[k] || h->held[k] == 0) continue;
    h->worker_solvers[k]->release();
    others -= h->held[k];
    h->held[k] = 0;
  }
  if (keep && others + after > h->budget && others + need <= h->budget) {
    keep = false;
    after = need;
  }
  if (others + after > h->budget && h->running > 0) return false;
  if (!keep && mine > 0) h->worker_solvers[idx]->release();
  h->held[idx] = after;
  return true;
}

static pins_status copy_problem(const pins_problem& p, OwnedProblem& o, std::string& why) {
  if (p.m < 1 || p.n < 1 || !p.a || !p.b) { why = "bad sizes or missing marginals"; return PINS_ERR_INVALID_ARG; }
  const cudaMemcpyKind k = p.on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  o.p = p;
  o.p.on_device = 0;
  o.a.resize(p.m); o.b.resize(p.n);
  cudaMemcpy(o.a.data(), p.a, sizeof(double) * p.m, k);
  cudaMemcpy(o.b.data(), p.b, sizeof(double) * p.n, k);
  o.p.a = o.a.data(); o.p.b = o.b.data();
  size_t mn = (size_t)p.m * p.n;
  if (p.kind == PINS_COST_DENSE_F64) {
    if (!p.C) { why = "dense cost requires C"; return PINS_ERR_INVALID_ARG; }
    o.C64.resize(mn); cudaMemcpy(o.C64.data(), p.C, sizeof(double) * mn, k); o.p.C = o.C64.data();
  } else if (p.kind == PINS_COST_DENSE_F32) {
    if (!p.C) { why = "dense cost requires C"; return PINS_ERR_INVALID_ARG; }
    o.C32.resize(mn); cudaMemcpy(o.C32.data(), p.C, sizeof(float) * mn, k); o.p.C = o.C32.data();
  } else if (p.kind == PINS_COST_POINTS_SQEUCLID) {
    if (!p.x || !p.y || p.d < 1 || p.d > 4) { why = "points cost requires x, y, 1 <= d <= 4"; return PINS_ERR_INVALID_ARG; }
    o.x.resize((size_t)p.m * p.d); o.y.resize((size_t)p.n * p.d);
    cudaMemcpy(o.x.data(), p.x, sizeof(double) * o.x.size(), k);
    cudaMemcpy(o.y.data(), p.y, sizeof(double) * o.y.size(), k);
    o.p.x = o.x.data(); o.p.y = o.y.data();
  }
  if (cudaGetLastError() != cudaSuccess) { why = "copying request inputs failed"; return PINS_ERR_INVALID_ARG; }
  return PINS_OK;
}

static void worker_main(pins_handle* h, int idx) {
  cudaSetDevice(h->device);
  Solver& solver = *h->worker_solvers[idx];
  for (;;) {
    std::shared_ptr<Job> job;
    {
      std::unique_lock<std::mutex> lk(h->mu);
      for (;;) {
        if (h->stopping) return;
        // admission by device memory (arrival order: the head waits for room)
        if (!h->queue.empty() && admit(h, idx, h->queue.front()->need)) {
          job = h->queue.front();
          h->queue.pop_front();
          h->busy[idx] = 1;
          ++h->running;
          break;
        }
        h->cv_work.wait(lk);
      }
    }
    job->prob.F.resize(job->prob.p.m);
    job->prob.G.resize(job->prob.p.n);
    job->res.F_out = job->prob.F.data();
    job->res.G_out = job->prob.G.data();
    pins_status st = solver.solve(h->cfg, job->prob.p, job->res);
    {
      std::lock_guard<std::mutex> lk(h->mu);
      job->status = st;
      job->error = solver.error();
      job->done = true;
      h->held[idx] = solver.arena_bytes();
      h->busy[idx] = 0;
      --h->running;
    }
    h->cv_done.notify_all();
    h->cv_work.notify_all();
  }
}

static void start_workers(pins_handle* h) {
  if (!h->workers.empty()) return;
  cudaSetDevice(h->device);
  for (int i = 0; i < h->cfg.max_inflight; ++i) {
    cudaStream_t s;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    h->worker_streams.push_back(s);
    h->worker_solvers.emplace_back(new Solver(h->device, h->sms, h->exp_table));
    h->worker_solvers.back()->set_stream(s);
    h->worker_solvers.back()->set_hooks(&h->hooks);
    h->held.push_back(0);
    h->busy.push_back(0);
  }
  for (int i = 0; i < h->cfg.max_inflight; ++i) h->workers.emplace_back(worker_main, h, i);
}

extern "C" pins_status pins_submit(pins_handle* h, const pins_problem* p, uint64_t* ticket) {
  if (!h || !p || !ticket) return PINS_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  auto job = std::make_shared<Job>();
  std::string why;
  pins_status s = copy_problem(*p, job->prob, why);
  if (s != PINS_OK) { set_error(h, why); return s; }
  job->need = job_need(h->cfg, job->prob.p);
  if (job->need > h->budget) { set_error(h, "request workspace exceeds the device memory budget"); return PINS_ERR_OOM; }
  {
    std::lock_guard<std::mutex> lk(h->mu);
    if ((int)h->queue.size() >= h->cfg.queue_capacity) { set_error(h, "queue full"); return PINS_ERR_QUEUE_FULL; }
    start_workers(h);
    job->ticket = h->next_ticket++;
    h->jobs[job->ticket] = job;
    h->queue.push_back(job);
    *ticket = job->ticket;
  }
  h->cv_work.notify_one();
  return PINS_OK;
}

static pins_status collect(pins_handle* h, std::shared_ptr<Job> job, pins_result* r) {
  double* F = r->F_out;
  double* G = r->G_out;
  *r = job->res;
  r->F_out = F; r->G_out = G;
  if (F) std::memcpy(F, job->prob.F.data(), sizeof(double) * job->prob.p.m);
  if (G) std::memcpy(G, job->prob.G.data(), sizeof(double) * job->prob.p.n);
  if (job->status != PINS_OK && !job->error.empty()) set_error(h, job->error);
  std::lock_guard<std::mutex> lk(h->mu);
  h->jobs.erase(job->ticket);
  return job->status;
}

extern "C" pins_status pins_poll(pins_handle* h, uint64_t ticket, pins_result* r) {
  if (!h || !r) return PINS_ERR_INVALID_ARG;
  std::shared_ptr<Job> job;
  {
    std::lock_guard<std::mutex> lk(h->mu);
    auto it = h->jobs.find(ticket);
    if (it == h->jobs.end()) return PINS_ERR_UNKNOWN_TICKET;
    if (!it->second->done) return PINS_ERR_PENDING;
    job = it->second;
  }
  return collect(h, job, r);
}

extern "C" pins_status pins_wait(pins_handle* h, uint64_t ticket, pins_result* r) {
  if (!h || !r) return PINS_ERR_INVALID_ARG;
  std::shared_ptr<Job> job;
  {
    std::unique_lock<std::mutex> lk(h->mu);
    auto it = h->jobs.find(ticket);
    if (it == h->jobs.end()) return PINS_ERR_UNKNOWN_TICKET;
    job = it->second;
    h->cv_done.wait(lk, [&] { return job->done; });
  }
  return collect(h, job, r);
}

extern "C" pins_status pins_solve_batch(pins_handle* h, const pins_problem* p, int count,
                                        pins_result* r) {
  if (!h || (!p && count > 0) || (!r && count > 0) || count < 0) return PINS_ERR_INVALID_ARG;
  std::vector<uint64_t> tickets(count, 0);
  std::vector<pins_status> sub(count, PINS_OK);
  pins_status first = PINS_OK;
  int i = 0;
  // submit in waves no larger than the queue so large batches never overflow it
  while (i < count) {
    int wave_end = std::min(count, i + h->cfg.queue_capacity);
    int wave_start = i;
    for (; i < wave_end; ++i) {
      sub[i] = pins_submit(h, p + i, &tickets[i]);
      if (sub[i] != PINS_OK) {
        std::memset(&r[i], 0, sizeof(pins_result));
        r[i].status = sub[i];
        if (first == PINS_OK) first = sub[i];
      }
    }
    for (int k = wave_start; k < wave_end; ++k) {
      if (sub[k] != PINS_OK) continue;
      pins_status s = pins_wait(h, tickets[k], &r[k]);
      if (s != PINS_OK && first == PINS_OK) first = s;
    }
  }
  return first;
}

// ------------------------------------------------------------------------- //
// step-level entry points (blocking, on the handle's stream)
// ------------------------------------------------------------------------- //
#define PINS_STEP_GUARD(h, p)                              \
  if (!(h) || !(p)) return PINS_ERR_INVALID_ARG;            \
  if (!(p)->on_device) { set_error(h, "step entry points take device pointers"); return PINS_ERR_INVALID_ARG; } \
  cudaSetDevice((h)->device)

static pins_status step_result(pins_handle* h, pins_status s) {
  if (s != PINS_OK) set_error(h, h->solver->error());
  return s;
}

extern "C" pins_status pins_step_sinkhorn(pins_handle* h, const pins_problem* p, double s,
                                          int iters, double* F, double* G, double* row_res) {
  PINS_STEP_GUARD(h, p);
  if (iters < 0 || !F || !G) return PINS_ERR_INVALID_ARG;
  return step_result(h, h->solver->step_sinkhorn(h->cfg, *p, s, iters, F, G, row_res));
}

extern "C" pins_status pins_step_marginals(pins_handle* h, const pins_problem* p, double s,
                                           const double* F, const double* G, double* r,
                                           double* c, double* out3) {
  PINS_STEP_GUARD(h, p);
  if (!F || !G || !r || !c || !out3) return PINS_ERR_INVALID_ARG;
  return step_result(h, h->solver->step_marginals(h->cfg, *p, s, F, G, r, c, out3));
}

extern "C" pins_status pins_step_sparsify(pins_handle* h, const pins_problem* p, double s,
                                          const double* F, const double* G, int keep,
                                          int* indptr, int* indices, double* data) {
  PINS_STEP_GUARD(h, p);
  if (!F || !G || !indptr || !indices || !data) return PINS_ERR_INVALID_ARG;
  return step_result(h, h->solver->step_sparsify(h->cfg, *p, s, F, G, keep, indptr, indices, data));
}

extern "C" pins_status pins_step_cg(pins_handle* h, int m, int n, double eta, const double* r,
                                    const double* c, const int* indptr, const int* indices,
                                    const double* data, int nnz, const double* rhs, double* d,
                                    double rtol, int max_iter, double* info) {
  if (!h || !r || !c || !indptr || !rhs || !d || !info) return PINS_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  return step_result(h, h->solver->step_cg(m, n, eta, r, c, indptr, indices, data, nnz, rhs, d,
                                           rtol, max_iter, info,
                                           h->cfg.prec == PINS_PREC_MIXED));
}

extern "C" pins_status pins_step_objective_increase(pins_handle* h, const pins_problem* p,
                                                    double s, const double* F, const double* G,
                                                    const double* df, const double* dg,
                                                    double alpha, double* out) {
  PINS_STEP_GUARD(h, p);
  if (!F || !G || !df || !dg || !out) return PINS_ERR_INVALID_ARG;
  return step_result(h, h->solver->step_objective_increase(h->cfg, *p, s, F, G, df, dg, alpha, out));
}

extern "C" pins_status pins_step_certificate(pins_handle* h, const pins_problem* p, double s,
                                             const double* F, const double* G, double* out6) {
  PINS_STEP_GUARD(h, p);
  if (!F || !G || !out6) return PINS_ERR_INVALID_ARG;
  return step_result(h, h->solver->step_certificate(h->cfg, *p, s, F, G, out6));
}

// ------------------------------------------------------------------------- //
// test hooks (host-side fault injection)
// ------------------------------------------------------------------------- //
extern "C" pins_status pins_test_inject_faults(pins_handle* h, int alloc_failures,
                                               int kernel_errors, int selection_failures) {
  if (!h || alloc_failures < 0 || kernel_errors < 0 || selection_failures < 0)
    return PINS_ERR_INVALID_ARG;
  h->hooks.alloc_fail.store(alloc_failures);
  h->hooks.kernel_error.store(kernel_errors);
  h->hooks.select_fail.store(selection_failures);
  return PINS_OK;
}

extern "C" pins_status pins_serving_held_bytes(pins_handle* h, size_t* held, size_t* budget) {
  if (!h || !held || !budget) return PINS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  size_t t = 0;
  for (size_t v : h->held) t += v;
  *held = t;
  *budget = h->budget;
  return PINS_OK;
}
