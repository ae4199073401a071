/*
 * pins.h -- C ABI of a GB300 (sm_103a) implementation of PINS: Proximal
 * Iterations with sparse Newton and Sinkhorn, for discrete Kantorovich optimal
 * transport (arXiv 2502.03749).
 *
 * Problem (Eq. ot, Section 1):
 *     min_X <C, X>   s.t.  X 1_n = a,  X^T 1_m = b,  X >= 0,
 * with a > 0, b > 0 and sum(a) = sum(b) = 1.
 *
 * Method (Algorithm 2, Section 3.2): an entropic proximal-point outer loop whose
 * k-th subproblem is entropic OT with the shifted cost C^k = C - eta log X^k
 * (Eq. eppa-sub); each subproblem is solved by a log-domain Sinkhorn warm-up and
 * damped Newton steps on a sparsified dual Hessian (CG + Armijo line search).
 * The library keeps X^k implicit as accumulated FP64 potentials:
 *     X~_ij = exp((F_i + G_j - s (C_ij + eta)) / eta),   s = k + 1,
 * so the cost is read or generated on the fly and never shifted in memory.
 *
 * Conventions for every call:
 *   - Matrices are row-major, 0-based; entry (i, j) of an m x n matrix is at
 *     i * n + j.  Vectors are contiguous.
 *   - "device pointer" means memory of the handle's CUDA device; "host pointer"
 *     means ordinary host memory.  pins_problem.on_device says which.
 *   - The caller owns every buffer it passes.  The library copies host inputs
 *     before a blocking call returns, and before pins_submit returns.
 *   - A call returns PINS_OK or an error status; pins_last_error() gives a
 *     one-line message for the last failing call on that handle.  Invalid input
 *     is rejected with PINS_ERR_INVALID_ARG before any device work starts.
 *   - There is no CPU fallback: if the CUDA device or kernels are unavailable
 *     the call fails with PINS_ERR_CUDA.
 */
#ifndef PINS_H_
#define PINS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pins_handle pins_handle;

typedef enum {
  PINS_OK = 0,
  PINS_ERR_INVALID_ARG = 1,   /* bad size, NaN, non-positive marginal, ... */
  PINS_ERR_OOM = 2,           /* device allocation failed */
  PINS_ERR_NOT_CONVERGED = 3, /* caps reached; result holds the last iterate */
  PINS_ERR_LINESEARCH = 4,    /* reserved: Armijo failures are recovered by a
                                 Sinkhorn step and counted, not returned */
  PINS_ERR_QUEUE_FULL = 5,    /* pins_submit: admission queue is full */
  PINS_ERR_PENDING = 6,       /* pins_poll: ticket not finished yet */
  PINS_ERR_CUDA = 7,          /* a CUDA runtime call or kernel failed */
  PINS_ERR_UNKNOWN_TICKET = 8 /* pins_poll: ticket never issued or already
                                 collected */
} pins_status;

/* How C is given (Section 5.2: "normalized so that all entries lie in [0,1]";
 * Section 3.2: the streaming implementation never materialises C). */
typedef enum {
  PINS_COST_DENSE_F64 = 0,      /* C: m*n doubles */
  PINS_COST_DENSE_F32 = 1,      /* C: m*n floats */
  PINS_COST_POINTS_SQEUCLID = 2,/* C_ij = cost_scale * |x_i - y_j|^2, x: m*d,
                                   y: n*d doubles (row-major, d = 1..4) */
  PINS_COST_GRID_SQEUCLID = 3   /* m = n = grid_s1 * grid_s2; pixel p =
                                   p1 * grid_s2 + p2; C_ij = cost_scale *
                                   ((i1-j1)^2 + (i2-j2)^2) */
} pins_cost_kind;

typedef enum {
  /* Every m x n pass in IEEE FP64 (FP64 exp).  The plain reference path. */
  PINS_PREC_FP64 = 0,
  /* m x n passes on the FP32 units: the Sinkhorn warm-up uses FP32 exp on a
   * double-float (compensated) exponent; the gradient, line-search, stopping and
   * certificate passes use a double-float table-driven exp (~1e-13 relative).
   * The CG keeps its vectors, matrix-vector product, inner products and step
   * lengths in double-float (about 48 significand bits) and checks the true residual
   * rhs - M x when its recurrence meets the tolerance.  Potentials, the outer
   * update and the stopping decisions stay FP64.  A dense FP64 cost is rounded
   * to FP32 once. */
  PINS_PREC_MIXED = 1
} pins_precision;

/* Solver settings.  pins_config_default() fills the hyperparameters of the
 * paper's Appendix E.1: eta = 1e-2, T1 = 100, T2 = 50, K = 250, Armijo beta =
 * 0.5 and c1 = 1e-4, CG relative residual 1e-6, marginal tolerance 1e-9, and the
 * Theorem 2 sparsity budget (gamma = 1: m + n - 1 kept coupling entries). */
typedef struct {
  double eta;           /* proximal/entropic parameter, > 0 */
  double tol_marg;      /* l1 marginal residual that ends an inner solve */
  double tol_gap;       /* certified relative gap that ends the outer loop;
                           0 disables the certificate test */
  double cg_rtol;       /* truncated-CG relative residual */
  double armijo_beta;   /* backtracking factor in (0, 1) */
  double armijo_c1;     /* sufficient-increase constant in (0, 1) */
  double sparsify_gamma;/* kept coupling entries = round(gamma (m + n - 1)) */
  int T1;               /* Sinkhorn warm-up cap per outer iteration */
  int T2;               /* Newton cap per outer iteration */
  int K;                /* outer (EPPA) cap */
  int max_cg;           /* CG iteration cap (also capped by m + n) */
  int max_backtrack;    /* Armijo halvings before the Sinkhorn fallback */
  int sinkhorn_check_every; /* warm-up residual check cadence (iterations) */
  int gap_every;        /* certificate cadence (outer iterations) */
  pins_precision prec;
  int device;           /* CUDA device ordinal */
  void* cuda_stream;    /* cudaStream_t for blocking calls; NULL = a stream
                           owned by the handle */
  int max_inflight;     /* serving: solves running at once (>= 1) */
  int queue_capacity;   /* serving: admitted-but-not-started requests */
  size_t device_mem_budget; /* serving: bytes of device workspace admission may
                               reserve; 0 = 80% of free memory at create time */
  int profile;          /* 1: time every kernel class of the blocking solver with
                           CUDA events (see pins_profile_read); 0 = off */
  int sparsify_one_pass; /* mixed path: 1 (default) selects the kept entries of the
                           later Newton steps of an outer iteration from the entries
                           above the previous threshold minus an adaptive margin (one
                           pass over C, exact top-K of the candidates); a failed
                           selection is redone by the histogram search.  0 = always
                           the histogram search.  The kept set is the same either way. */
} pins_config;

typedef struct {
  pins_cost_kind kind;
  int m, n;             /* marginal sizes (>= 1) */
  int d;                /* point dimension for POINTS (1..4), else ignored */
  const void* C;        /* DENSE_*: m*n entries; else NULL */
  const double* x;      /* POINTS: m*d */
  const double* y;      /* POINTS: n*d */
  double cost_scale;    /* POINTS, GRID: multiplies the squared distance */
  int grid_s1, grid_s2; /* GRID */
  const double* a;      /* m, positive, sums to 1 */
  const double* b;      /* n, positive, sums to 1 */
  int on_device;        /* 1: every pointer above is a device pointer */
} pins_problem;

typedef struct {
  pins_status status;
  double cost;          /* <C, X~> of the final plan (unrounded, as reported
                           against the LP optimum in Section 5) */
  double cost_ub;       /* cost of the plan rounded onto the transport polytope
                           (Altschuler-Weed-Rigollet), >= OPT */
  double dual_lb;       /* LP dual bound, <= OPT: the larger of the c-transform
                           bounds of the entropic dual and of the support-tree
                           dual (see pins_step_certificate) */
  double rel_gap;       /* (cost_ub - dual_lb) / dual_lb */
  double marg_resid_l1; /* ||X~1 - a||_1 + ||X~^T 1 - b||_1 of the final plan */
  double s;             /* final scale: the plan is exp((F+G-s(C+eta))/eta) */
  int outer_iters, sinkhorn_iters, newton_iters, cg_iters, ls_trials,
      ls_failures, gpu_launches;
  double seconds;       /* wall time of the solve inside the library */
  double* F_out;        /* optional caller buffer (host memory), m doubles */
  double* G_out;        /* optional caller buffer (host memory), n doubles */
} pins_result;

/* Fills *cfg with the paper's defaults (Appendix E.1). */
void pins_config_default(pins_config* cfg);

/* Creates a handle on cfg->device.  Allocates no per-problem memory yet.
 * Errors: PINS_ERR_INVALID_ARG (cfg or out NULL, bad values), PINS_ERR_CUDA. */
pins_status pins_create(const pins_config* cfg, pins_handle** out);

/* Frees every resource of the handle; waits for running solves first. */
void pins_destroy(pins_handle* h);

/* One-line description of the last error on this handle ("" if none). */
const char* pins_last_error(pins_handle* h);

/* Blocking solve of one problem (Algorithm 2) on the handle's stream.
 * Result fields are filled on PINS_OK and PINS_ERR_NOT_CONVERGED.  With
 * cfg.profile = 0, each block of sinkhorn_check_every warm-up iterations is
 * captured once per outer iteration (thread-local capture mode on that stream)
 * and launched as one CUDA graph; where capture is not possible the kernels
 * are launched one by one.  Both give the same result. */
pins_status pins_solve(pins_handle* h, const pins_problem* p, pins_result* r);

/* Blocking solve of count independent problems.  Instances run concurrently on
 * the device (one stream per in-flight instance); each result equals the result
 * of pins_solve on that problem alone.  Returns the first non-OK status, with
 * every r[i].status filled. */
pins_status pins_solve_batch(pins_handle* h, const pins_problem* p, int count,
                             pins_result* r);

/* Serving: admits a request (inputs are copied before return) and returns a
 * ticket.  Requests run as device memory and in-flight slots free up, overlapped
 * on the device.  Errors: PINS_ERR_QUEUE_FULL, PINS_ERR_INVALID_ARG.
 * Each slot has its own stream.  The CUDA runtime maps streams onto
 * CUDA_DEVICE_MAX_CONNECTIONS hardware work queues (8 unless the environment
 * says otherwise, read when the process first uses CUDA); with more slots than
 * queues, a short request's kernels can wait behind a long one's in a shared
 * queue, so a server sets it to at least max_inflight (32 at most). */
pins_status pins_submit(pins_handle* h, const pins_problem* p, uint64_t* ticket);

/* Serving: PINS_ERR_PENDING while the ticket runs; otherwise fills *r (F_out and
 * G_out, if set in *r, receive the potentials), releases the ticket and returns
 * the solve status. */
pins_status pins_poll(pins_handle* h, uint64_t ticket, pins_result* r);

/* Serving: blocks until the ticket finishes, then behaves as pins_poll. */
pins_status pins_wait(pins_handle* h, uint64_t ticket, pins_result* r);

/* Profiling of the blocking solver (pins_solve and the step entry points) when
 * the handle was created with cfg.profile = 1.  Each kernel launch is bracketed
 * by CUDA events on the solver's stream; durations are accumulated per class.
 * pins_profile_read copies min(n, pins_profile_classes()) entries of device
 * milliseconds (ms) and launch counts (launches; either may be NULL), then
 * clears the totals if reset != 0.  Classes: 0 row_lse, 1 col_lse,
 * 2 marginals, 3 trial, 4 key_hist, 5 key_compact, 6 select, 7 csr_write,
 * 8 csc, 9 cg, 10 certificate, 11 vector. */
int pins_profile_classes(void);
const char* pins_profile_name(int k);
pins_status pins_profile_read(pins_handle* h, double* ms, long long* launches, int n,
                              int reset);

/* ------------------------------------------------------------------------- */
/* Step-level entry points.  Each runs one hot-path step on device pointers,  */
/* on the handle's stream, and returns after the step completes.  They expose */
/* the kernels the solver uses so each step can be checked on its own.        */
/* p->on_device must be 1.  F, G are FP64 accumulated potentials (length m,   */
/* n); s is the outer scale k + 1.  The handle's cfg.prec selects the kernels.*/
/* ------------------------------------------------------------------------- */

/* Sinkhorn warm-up half-steps (Algorithm 2, warm-up loop; Algorithm 1 in log
 * form): `iters` Gauss-Seidel iterations, each F_i <- eta log a_i - eta LSE_j(
 * (G_j - s (C_ij + eta)) / eta), then G_j likewise with the new F.  F, G are
 * updated in place.  row_res (device, may be NULL) receives, per iteration, the
 * l1 row residual measured by that iteration's row half-step. */
pins_status pins_step_sinkhorn(pins_handle* h, const pins_problem* p, double s,
                               int iters, double* F, double* G, double* row_res);

/* Row and column sums of X~ (gradient formulas after Eq. eppa-sub-dual):
 * r (m), c (n) device outputs; out3 (device, 3 doubles) = {l1 residual,
 * sum X~, max_ij (F_i + G_j - s (C_ij + eta))}. */
pins_status pins_step_marginals(pins_handle* h, const pins_problem* p, double s,
                                const double* F, const double* G, double* r,
                                double* c, double* out3);

/* Sparsify (Algorithm 2; Section 3.2; Theorem 2): keeps the `keep` largest
 * entries of X~ ranked by F_i + G_j - s (C_ij + eta) (FP64 path; the FP32 value
 * of log X~ on the mixed path), ties to the lower row-major index, and writes
 * them as CSR: indptr (m + 1), indices (keep), data (keep, X~_ij), all device
 * pointers.  keep must be in [1, m*n]. */
pins_status pins_step_sparsify(pins_handle* h, const pins_problem* p, double s,
                               const double* F, const double* G, int keep,
                               int* indptr, int* indices, double* data);

/* Truncated Jacobi-preconditioned CG on M d = rhs with
 * M = (1/eta) [[diag r, S], [S^T, diag c]] (the negated sparsified Hessian of
 * Eq. eq:eppa-hess).  S is CSR (indptr m+1, indices/data nnz).  rhs, d: m + n
 * device doubles.  info (device, 2 doubles) = {iterations, relative residual}.
 * On a PINS_PREC_FP64 handle every operation is FP64.  On a PINS_PREC_MIXED
 * handle the vectors, the matrix-vector product, the inner products and the
 * step lengths are kept in double-float (FP32 pairs, ~48 significand bits), in
 * the single-reduction ordering that gives the textbook PCG's iterates in exact
 * arithmetic (its iteration count within a few per cent); when the recurrence
 * residual meets rtol, the true residual rhs - M d is formed and, if it is
 * above 2 rtol ||rhs||, the iteration restarts from d (at most three times).
 * info[1] is then the last measured ||r|| / ||rhs||. */
pins_status pins_step_cg(pins_handle* h, int m, int n, double eta,
                         const double* r, const double* c, const int* indptr,
                         const int* indices, const double* data, int nnz,
                         const double* rhs, double* d, double rtol, int max_iter,
                         double* info);

/* Objective increase for the Armijo test (Algorithm 2 line search):
 * out (device, 1 double) = P(x + alpha d) - P(x) = alpha (<a,df> + <b,dg>)
 *   - eta sum_ij X~_ij expm1(alpha (df_i + dg_j) / eta);  -inf on overflow.
 * A PINS_PREC_MIXED handle evaluates the equal form alpha (<a - r, df> +
 * <b - c, dg>) - eta sum_ij X~_ij (expm1(t_ij) - t_ij), t_ij = alpha (df_i +
 * dg_j) / eta, with r, c the marginals of X~: its terms do not cancel, so the
 * nonnegative sum is taken in FP32. */
pins_status pins_step_objective_increase(pins_handle* h, const pins_problem* p,
                                         double s, const double* F,
                                         const double* G, const double* df,
                                         const double* dg, double alpha,
                                         double* out);

/* Certificate of the stopping test (the outer stop of Algorithm 2; the bracket
 * [LB, UB] bounds the relative error to the LP optimum that Section 5 reports):
 * out6 (device, 6 doubles) = {<C, X~>, UB = <C, round(X~)>
 * (Altschuler-Weed-Rigollet rounding), LB, relative gap (UB - LB) / LB,
 * LB_entropic, LB_tree}.  LB = max(LB_entropic, LB_tree), each the double
 * c-transform bound <a, u'> + <b, v> of a row potential: LB_entropic from
 * u = F/s - eta; LB_tree from the support-tree dual, i.e. potentials tight
 * (u_i + v_j = C_ij) on the maximum-weight spanning forest of the
 * 2(m + n - 1) largest entries of X~ (ranked by F_i + G_j - s (C_ij + eta),
 * ties to the lower row-major index; each tree's lowest node, rows first,
 * keeps its entropic potential).  Both are valid LP lower bounds for any F, G;
 * LB_tree reaches OPT once the plan has concentrated on an optimal basis. */
pins_status pins_step_certificate(pins_handle* h, const pins_problem* p,
                                  double s, const double* F, const double* G,
                                  double* out6);

/* Serving: device bytes the worker pool's arenas hold (reserved for running
 * requests plus arenas idle workers keep for reuse) and the admission budget.
 * Admission keeps *held <= *budget, except for a single request running alone.
 * The handle's own blocking solver (pins_solve, step entry points) is outside
 * this pool.  The paper has no counterpart: it is serving bookkeeping. */
pins_status pins_serving_held_bytes(pins_handle* h, size_t* held, size_t* budget);

/* Test hook (the paper has no counterpart): host-side fault injection on this
 * handle's solvers, so that error paths are tested without faulting a GPU.
 * The next `alloc_failures` workspace allocations report failure before any
 * device allocation is attempted (the solve returns PINS_ERR_OOM); the next
 * `kernel_errors` line-search checks of the kernels' error word see an error
 * bit (the solve returns PINS_ERR_CUDA); the next `selection_failures`
 * one-pass selections of the mixed path read as failed, so their Newton steps
 * are redone with the histogram search (the result is unchanged).  Counters
 * are consumed across all of the handle's solvers (blocking and serving);
 * zeros clear them.  Errors: PINS_ERR_INVALID_ARG for a NULL handle or
 * negative counts. */
pins_status pins_test_inject_faults(pins_handle* h, int alloc_failures, int kernel_errors,
                                    int selection_failures);

/* ------------------------------------------------------------------------- */
/* Allocation-free marginal pass.  The paper has no counterpart: this entry   */
/* serves callers that cannot allocate device memory (a host framework that   */
/* owns all device memory through its own pool, a real-time loop that must    */
/* not enter the driver's allocator, an embedding that reserves everything at */
/* start-up).                                                                 */
/* ------------------------------------------------------------------------- */
#define PINS_NOALLOC_MAX_DIM 4096
#define PINS_NOALLOC_SCRATCH_BYTES (3584u * 1024u)

/* Same result as pins_step_marginals (row sums r, column sums c of the plan
 * exp((F_i + G_j - s (C_ij + eta)) / eta); out3 = {l1 marginal residual, sum of
 * the plan, max_ij (F_i + G_j - s (C_ij + eta))}), without a handle and without
 * allocating: its scratch is a fixed static device array of
 * PINS_NOALLOC_SCRATCH_BYTES that each GPU loading the library keeps until exit.
 * Every pointer (p's arrays, F, G, r, c, out3) is a device pointer of the
 * current device.  prec is PINS_PREC_FP64 (cost kinds DENSE_F64, POINTS, GRID)
 * or PINS_PREC_MIXED (DENSE_F32, POINTS, GRID).  The work is queued on
 * cuda_stream (NULL: the legacy default stream) and the call returns without
 * waiting.  The first call on a device sets up that device's scratch (a symbol
 * lookup and a small host-to-device copy): make it before any stream capture.
 * All calls on a device share its scratch, so calls that overlap on the GPU
 * race; order them on one stream.  Returns PINS_ERR_INVALID_ARG if m or n
 * exceeds PINS_NOALLOC_MAX_DIM or an argument is invalid, PINS_ERR_CUDA if a
 * CUDA call fails. */
pins_status pins_marginals_noalloc(const pins_problem* p, double eta, int prec, double s,
                                   const double* F, const double* G, double* r, double* c,
                                   double* out3, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PINS_H_ */
