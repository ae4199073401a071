// Host-side solver of one PINS instance on one CUDA stream (Algorithm 2).
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <string>
#include <vector>
#include "../../include/pins.h"
#include "pins_kernels.h"
#include "pins_sparsify.cuh"

namespace pins {

// Device workspace of one instance (one arena, carved in fixed order).
struct Workspace {
  size_t bytes = 0;
  void* base = nullptr;
  int m = 0, n = 0, kcap = 0, t1cap = 0;
  // potentials and vectors (FP64)
  double *F, *G, *Phi, *Psi, *A64, *B64, *r, *c, *rt, *ct, *Pt64, *Qt64;
  double *grad, *dir, *cg_res, *cg_p, *cg_q, *ab;
  double* lab;                                  // (log a; log b): mixed grid half-steps
  double *xs, *u, *rr, *cr, *cp, *tc, *u2, *ys, *ec, *c1, *v;
  double *uT, *vT, *u2T;   // support-tree dual of the certificate
  TreeWS tw;
  float2 *Add, *Bdd;
  MergeWS mws;
  SparsifyState* st;
  unsigned int* hist;
  double* cand_key; long long* cand_idx;
  SparseWS sw;
  int* ent_tgt; float2* ent_val; int* ent_row;   // double-float CG: packed entries (2 kcap)
  float* fkey; unsigned long long* fij;          // one-pass selection candidates
  float* cg_u;                                  // double-float CG: u exchange (m + n)
  double* cg_part;
  double* scal;            // device scalars (see Solver::SC_*)
  // uploaded inputs
  double *a, *b, *C64, *x, *y;
  float *C32, *xf, *yf;
};

size_t workspace_bytes(int m, int n, int kcap, int t1cap, int cost_kind, bool mixed,
                       bool host_inputs, int d);
// kept-entry capacity of a full solve: the Newton steps' gamma (m + n - 1) and
// the certificate's 2 (m + n - 1), at most m n
int solve_kcap(const pins_config& cfg, int m, int n);
// device bytes pins_solve needs for problem p (host inputs)
size_t solve_workspace_bytes(const pins_config& cfg, const pins_problem& p);

// Host-side fault injection for tests: no GPU fault is ever caused.  alloc_fail
// makes the next workspace allocations report failure before any cudaMalloc;
// kernel_error makes the next line-search syncs report a kernel error flag;
// select_fail makes the next one-pass selections read as failed, so the step is
// redone by the histogram search.
struct FaultHooks {
  std::atomic<int> alloc_fail{0};
  std::atomic<int> kernel_error{0};
  std::atomic<int> select_fail{0};
};

class Solver {
 public:
  // scalar slots in Workspace::scal (doubles)
  // (SC_STATE: 12 doubles of pinned host memory receive the SparsifyState)
  enum { SC_MARG = 0, SC_TRIAL = 4, SC_DOTS = 8, SC_CERT = 12, SC_CG = 16, SC_STATE = 18,
         SC_FLAG = 30, SC_FAST = 32, SC_CERT2 = 36, SC_ROWRES = 40 };

  Solver(int device, int sms, const float2* exp_table);
  ~Solver();
  Solver(const Solver&) = delete;
  Solver& operator=(const Solver&) = delete;

  void set_stream(cudaStream_t s) { stream_ = s; }
  void set_hooks(FaultHooks* f) { hooks_ = f; }
  cudaStream_t stream() const { return stream_; }
  size_t arena_bytes() const { return ws_.bytes; }
  void release();

  // Full solve.  cfg is read-only; r is filled.
  pins_status solve(const pins_config& cfg, const pins_problem& p, pins_result& r);

  // step-level entry points (device pointers, p.on_device == 1)
  pins_status step_sinkhorn(const pins_config& cfg, const pins_problem& p, double s, int iters,
                            double* F, double* G, double* row_res);
  pins_status step_marginals(const pins_config& cfg, const pins_problem& p, double s,
                             const double* F, const double* G, double* r, double* c,
                             double* out3);
  pins_status step_sparsify(const pins_config& cfg, const pins_problem& p, double s,
                            const double* F, const double* G, int keep, int* indptr,
                            int* indices, double* data);
  pins_status step_cg(int m, int n, double eta, const double* r, const double* c,
                      const int* indptr, const int* indices, const double* data, int nnz,
                      const double* rhs, double* d, double rtol, int max_iter, double* info,
                      bool mixed);
  pins_status step_objective_increase(const pins_config& cfg, const pins_problem& p, double s,
                                      const double* F, const double* G, const double* df,
                                      const double* dg, double alpha, double* out);
  pins_status step_certificate(const pins_config& cfg, const pins_problem& p, double s,
                               const double* F, const double* G, double* out6);

  const std::string& error() const { return err_; }
  // the CG of one Newton step (double-float cluster kernel on the mixed path when
  // it fits, else the FP64 kernels).  rhs == NULL: rhs = (a - r; b - c).  dots
  // (may be NULL) receives <rhs, d> and <ab, d>.
  cudaError_t run_cg(bool mixed, int m, int n, double eta, const double* r, const double* c,
                     const int* indptr, const int* indices, const double* data, int nnz,
                     const double* rhs, double* d, double rtol, int max_iter, double* info,
                     const double* ab, double* dots);
  long long launches() const { return launches_; }

  // Optional per-kernel-class device timing: CUDA events recorded on the
  // solver's stream around each launch, drained at every host sync.
  enum { PC_ROW_LSE = 0, PC_COL_LSE, PC_MARG, PC_TRIAL, PC_HIST, PC_COMPACT, PC_SELECT,
         PC_WRITE, PC_CSC, PC_CG, PC_CERT, PC_VEC, PC_COUNT };
  static const char* prof_name(int k);
  void set_profile(bool on) { profile_ = on; }
  void prof_read(double* ms, long long* cnt, int n, bool reset);

 private:
  void prof_begin(int cls);
  void prof_end();
  void prof_drain();
  bool profile_ = false;
  std::vector<cudaEvent_t> ev_pool_;
  std::vector<std::pair<int, int>> ev_pending_;   // (class, index of start event)
  int ev_next_ = 0, ev_cls_ = -1;
  double prof_ms_[PC_COUNT] = {};
  long long prof_cnt_[PC_COUNT] = {};

  pins_status prepare(const pins_config& cfg, const pins_problem& p, bool need_kcap);
  pins_status ensure(int m, int n, int kcap, int t1cap, int kind, bool mixed, bool host_in, int d);
  pins_status upload(const pins_problem& p);
  pins_status check(const char* where);
  pins_status sync(const char* where);
  void prep(double s);
  // with_res: also form the row residual into SC_ROWRES + t (else skipped)
  void sinkhorn_iter(double s, int t, bool with_res = true);
  void marg(double s, bool trial, double alpha = 0.0);
  pins_status sparsify(double s, int keep, double zmax, int* nnz_out, bool csc = true);
  // one-pass selection for the later Newton steps of an outer iteration (mixed);
  // launches only, the outcome is read at the next line-search sync
  void sparsify_fast(double s, int keep, float tau_guess);
  // certificate at (F, G, s); zmax = max_ij z at that point (window of the
  // support selection of the tree dual)
  pins_status certificate(double s, double zmax);
  PassArgs args(double s, const double* F, const double* G);

  int device_, sms_;
  const float2* exp_table_;
  FaultHooks* hooks_ = nullptr;
  cudaStream_t stream_ = nullptr;
  Workspace ws_;
  double* h_scal_ = nullptr;   // pinned mirror of ws_.scal
  int h_scal_len_ = 0;
  std::string err_;
  long long launches_ = 0;
  // per-problem state
  const PassSet* ps_ = nullptr;
  CostArgs cost_{};
  int m_ = 0, n_ = 0;
  double eta_ = 0;
  bool mixed_ = false;
  TileGeom geom_{};
  const double* a_ = nullptr;
  const double* b_ = nullptr;
};

}  // namespace pins
