// Host driver of Algorithm 2 on one CUDA stream.  All m x n and vector work runs
// in the kernels of pins_kernels_*.cu / pins_sparse.cu / pins_select.cu; the host
// only sequences launches and reads a few scalars back to take the decisions the
// algorithm makes (warm-up exit, Newton stop, Armijo acceptance, outer stop).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include "pins_solver.h"

namespace pins {

namespace {

struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <class T> T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += std::max<size_t>(count, 1) * sizeof(T);
    return p;
  }
};

int kind_of(pins_cost_kind k) {
  switch (k) {
    case PINS_COST_DENSE_F64:
    case PINS_COST_DENSE_F32: return COST_DENSE;
    case PINS_COST_POINTS_SQEUCLID: return COST_POINTS;
    case PINS_COST_GRID_SQEUCLID: return COST_GRID;
  }
  return -1;
}

struct InputPlan {   // which converted input copies an instance needs
  bool c64 = false, c32 = false, xy64 = false, xy32 = false, ab = false;
};

InputPlan plan_inputs(pins_cost_kind kind, bool mixed, bool host_in) {
  InputPlan q;
  q.ab = host_in;
  if (kind == PINS_COST_DENSE_F64) {
    if (!mixed) q.c64 = host_in;
    else { q.c32 = true; q.c64 = host_in; }            // host: staged then converted
  } else if (kind == PINS_COST_DENSE_F32) {
    if (!mixed) { q.c64 = true; q.c32 = host_in; }     // widened once
    else q.c32 = host_in;
  } else if (kind == PINS_COST_POINTS_SQEUCLID) {
    q.xy64 = host_in;
    q.xy32 = mixed;
  }
  return q;
}

void carve(Carver& cv, Workspace& w, int m, int n, int kcap, int t1cap, const TileGeom& g,
           const InputPlan& ip, size_t mn, int d) {
  const int N = m + n;
  w.F = cv.take<double>(m); w.G = cv.take<double>(n);
  w.Phi = cv.take<double>(m); w.Psi = cv.take<double>(n);
  w.A64 = cv.take<double>(m); w.B64 = cv.take<double>(n);
  w.r = cv.take<double>(m); w.c = cv.take<double>(n);
  w.rt = cv.take<double>(m); w.ct = cv.take<double>(n);
  w.Pt64 = cv.take<double>(m); w.Qt64 = cv.take<double>(n);
  w.grad = cv.take<double>(N); w.dir = cv.take<double>(N);
  w.lab = cv.take<double>(N);
  w.cg_res = cv.take<double>(N); w.cg_p = cv.take<double>(N); w.cg_q = cv.take<double>(2 * (size_t)N);
  w.ab = cv.take<double>(N);
  w.xs = cv.take<double>(m); w.u = cv.take<double>(m); w.rr = cv.take<double>(m);
  w.cr = cv.take<double>(m); w.cp = cv.take<double>(m); w.tc = cv.take<double>(m);
  w.u2 = cv.take<double>(m);
  w.ys = cv.take<double>(n); w.ec = cv.take<double>(n); w.c1 = cv.take<double>(n);
  w.v = cv.take<double>(n);
  w.uT = cv.take<double>(m); w.u2T = cv.take<double>(m); w.vT = cv.take<double>(n);
  w.tw.erow = cv.take<int>(kcap); w.tw.okey = cv.take<unsigned long long>(kcap);
  w.tw.eflag = cv.take<int>(kcap);
  w.tw.comp = cv.take<int>(N); w.tw.bkey = cv.take<unsigned long long>(N);
  w.tw.be = cv.take<int>(N); w.tw.lvl = cv.take<int>(N); w.tw.minid = cv.take<int>(N);
  w.tw.pot = cv.take<double>(N);
  w.Add = cv.take<float2>(m); w.Bdd = cv.take<float2>(n);
  w.mws.rowpart0 = cv.take<double>((size_t)g.gx * m);
  w.mws.rowpart1 = cv.take<double>((size_t)g.gx * m);
  w.mws.rowpart2 = cv.take<double>((size_t)g.gx * m);
  w.mws.rowpart3 = cv.take<double>((size_t)g.gx * m);
  w.mws.rowpart4 = cv.take<double>((size_t)g.gx * m);
  w.mws.rowpart5 = cv.take<double>((size_t)g.gx * m);
  w.mws.colpart0 = cv.take<double>((size_t)g.gy * n);
  w.mws.colpart1 = cv.take<double>((size_t)g.gy * n);
  w.mws.colpart2 = cv.take<double>((size_t)g.gy * n);
  w.mws.scal_row = cv.take<double>(8 * PINS_GY_MAX);
  w.mws.scal_col = cv.take<double>(4 * PINS_GX_MAX * PINS_GY_MAX + PINS_GX_MAX);
  w.mws.cnt_row = cv.take<unsigned int>(PINS_ROW_GROUPS);
  w.mws.cnt_col = cv.take<unsigned int>(PINS_GX_MAX);
  w.mws.cnt_all = cv.take<unsigned int>(1);
  w.st = cv.take<SparsifyState>(1);
  w.hist = cv.take<unsigned int>(PINS_HIST_NB + 1);
  w.cand_key = cv.take<double>(PINS_CAND_CAP); w.cand_idx = cv.take<long long>(PINS_CAND_CAP);
  w.sw.rowcnt = cv.take<int>(m); w.sw.colcnt = cv.take<int>(n);
  w.sw.indptr = cv.take<int>(m + 1); w.sw.indices = cv.take<int>(kcap);
  w.sw.data = cv.take<double>(kcap);
  w.sw.colptr = cv.take<int>(n + 1); w.sw.rowidx = cv.take<int>(kcap);
  w.sw.cdata = cv.take<double>(kcap);
  w.sw.trow = cv.take<int>(kcap); w.sw.tval = cv.take<double>(kcap);
  w.sw.tcol = cv.take<int>(kcap); w.sw.tcval = cv.take<double>(kcap);
  w.sw.longseg = cv.take<int>(N); w.sw.nlong = cv.take<int>(1);
  w.fkey = cv.take<float>(PINS_FAST_CAP); w.fij = cv.take<unsigned long long>(PINS_FAST_CAP);
  w.ent_tgt = cv.take<int>(2 * (size_t)kcap + PINS_DDCG_ENTRY_PAD);
  w.ent_val = cv.take<float2>(2 * (size_t)kcap + PINS_DDCG_ENTRY_PAD);
  w.ent_row = cv.take<int>(2 * (size_t)kcap + PINS_DDCG_ENTRY_PAD);
  w.cg_u = cv.take<float>(4 * (size_t)N);   // two buffers of N double-float pairs
  w.cg_part = cv.take<double>(3 * 64 + 8);
  w.scal = cv.take<double>(Solver::SC_ROWRES + t1cap + 8);
  w.a = ip.ab ? cv.take<double>(m) : nullptr;
  w.b = ip.ab ? cv.take<double>(n) : nullptr;
  w.C64 = ip.c64 ? cv.take<double>(mn) : nullptr;
  w.C32 = ip.c32 ? cv.take<float>(mn) : nullptr;
  w.x = ip.xy64 ? cv.take<double>((size_t)m * d) : nullptr;
  w.y = ip.xy64 ? cv.take<double>((size_t)n * d) : nullptr;
  w.xf = ip.xy32 ? cv.take<float>((size_t)m * d) : nullptr;
  w.yf = ip.xy32 ? cv.take<float>((size_t)n * d) : nullptr;
}

}  // namespace

size_t workspace_bytes(int m, int n, int kcap, int t1cap, int cost_kind, bool mixed,
                       bool host_inputs, int d) {
  Workspace w;
  Carver cv(nullptr);
  TileGeom g = make_geom(m, n);
  InputPlan ip = plan_inputs((pins_cost_kind)cost_kind, mixed, host_inputs);
  carve(cv, w, m, n, kcap, t1cap, g, ip, (size_t)m * n, d < 1 ? 1 : d);
  return cv.off + 256;
}

int solve_kcap(const pins_config& cfg, int m, int n) {
  const long long ksup = 2LL * (m + n - 1);
  const long long kg = llround(cfg.sparsify_gamma * (m + n - 1));
  return (int)std::min<long long>((long long)m * n, std::max({1LL, ksup, kg}));
}

size_t solve_workspace_bytes(const pins_config& cfg, const pins_problem& p) {
  return workspace_bytes(p.m, p.n, solve_kcap(cfg, p.m, p.n), std::max(cfg.T1, 1), p.kind,
                         cfg.prec == PINS_PREC_MIXED, true, p.d);
}

Solver::Solver(int device, int sms, const float2* exp_table)
    : device_(device), sms_(sms), exp_table_(exp_table) {}

Solver::~Solver() { release(); }

const char* Solver::prof_name(int k) {
  static const char* names[PC_COUNT] = {"row_lse", "col_lse", "marginals", "trial", "key_hist",
                                        "key_compact", "select", "csr_write", "csc", "cg",
                                        "certificate", "vector"};
  return (k >= 0 && k < PC_COUNT) ? names[k] : "";
}

void Solver::prof_begin(int cls) {
  if (!profile_) return;
  while ((int)ev_pool_.size() < ev_next_ + 2) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    ev_pool_.push_back(e);
  }
  cudaEventRecord(ev_pool_[ev_next_], stream_);
  ev_pending_.push_back(std::make_pair(cls, ev_next_));
  ev_next_ += 2;
}

void Solver::prof_end() {
  if (!profile_ || ev_pending_.empty()) return;
  cudaEventRecord(ev_pool_[ev_pending_.back().second + 1], stream_);
}

void Solver::prof_drain() {
  for (auto& pr : ev_pending_) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev_pool_[pr.second], ev_pool_[pr.second + 1]) == cudaSuccess) {
      prof_ms_[pr.first] += ms;
      prof_cnt_[pr.first] += 1;
    }
  }
  cudaGetLastError();
  ev_pending_.clear();
  ev_next_ = 0;
}

void Solver::prof_read(double* ms, long long* cnt, int n, bool reset) {
  for (int k = 0; k < n && k < PC_COUNT; ++k) {
    if (ms) ms[k] = prof_ms_[k];
    if (cnt) cnt[k] = prof_cnt_[k];
  }
  if (reset)
    for (int k = 0; k < PC_COUNT; ++k) { prof_ms_[k] = 0.0; prof_cnt_[k] = 0; }
}

void Solver::release() {
  for (auto e : ev_pool_) cudaEventDestroy(e);
  ev_pool_.clear();
  ev_pending_.clear();
  ev_next_ = 0;
  if (ws_.base) cudaFree(ws_.base);
  ws_ = Workspace();
  if (h_scal_) cudaFreeHost(h_scal_);
  h_scal_ = nullptr;
  h_scal_len_ = 0;
}

pins_status Solver::check(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    err_ = std::string(where) + ": " + cudaGetErrorString(e);
    return PINS_ERR_CUDA;
  }
  return PINS_OK;
}

pins_status Solver::sync(const char* where) {
  cudaError_t e = cudaStreamSynchronize(stream_);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    err_ = std::string(where) + ": " + cudaGetErrorString(e);
    return PINS_ERR_CUDA;
  }
  if (profile_) prof_drain();
  return PINS_OK;
}

pins_status Solver::ensure(int m, int n, int kcap, int t1cap, int kind, bool mixed, bool host_in,
                           int d) {
  size_t need = workspace_bytes(m, n, kcap, t1cap, kind, mixed, host_in, d);
  if (!ws_.base || need > ws_.bytes) {
    if (ws_.base) { cudaFree(ws_.base); ws_.base = nullptr; ws_.bytes = 0; }
    void* p = nullptr;
    const bool injected = hooks_ && hooks_->alloc_fail.load() > 0 &&
                          hooks_->alloc_fail.fetch_sub(1) > 0;
    if (injected) {
      err_ = "device allocation of " + std::to_string(need) + " bytes failed (injected)";
      return PINS_ERR_OOM;
    }
    if (cudaMalloc(&p, need) != cudaSuccess) {
      cudaGetLastError();
      err_ = "device allocation of " + std::to_string(need) + " bytes failed";
      return PINS_ERR_OOM;
    }
    ws_.base = p;
    ws_.bytes = need;
  }
  Carver cv(ws_.base);
  size_t bytes = ws_.bytes;
  void* base = ws_.base;
  TileGeom g = make_geom(m, n);
  carve(cv, ws_, m, n, kcap, t1cap, g, plan_inputs((pins_cost_kind)kind, mixed, host_in),
        (size_t)m * n, d < 1 ? 1 : d);
  ws_.base = base; ws_.bytes = bytes;
  ws_.m = m; ws_.n = n; ws_.kcap = kcap; ws_.t1cap = t1cap;
  // counters start at zero; every kernel leaves them at zero
  cudaMemsetAsync(ws_.mws.cnt_row, 0, sizeof(unsigned int) * PINS_ROW_GROUPS, stream_);
  cudaMemsetAsync(ws_.mws.cnt_col, 0, sizeof(unsigned int) * PINS_GX_MAX, stream_);
  cudaMemsetAsync(ws_.mws.cnt_all, 0, sizeof(unsigned int), stream_);
  cudaMemsetAsync(ws_.hist, 0, sizeof(unsigned int) * (PINS_HIST_NB + 1), stream_);
  cudaMemsetAsync(ws_.sw.colcnt, 0, sizeof(int) * n, stream_);
  int len = SC_ROWRES + t1cap + 8;
  if (len > h_scal_len_) {
    if (h_scal_) cudaFreeHost(h_scal_);
    if (cudaMallocHost(&h_scal_, sizeof(double) * len) != cudaSuccess) {
      h_scal_ = nullptr; h_scal_len_ = 0;
      err_ = "pinned host allocation failed";
      return PINS_ERR_OOM;
    }
    h_scal_len_ = len;
  }
  return check("workspace");
}

static bool vec_ok(const double* v, int len, double& sum) {
  sum = 0.0;
  for (int i = 0; i < len; ++i) {
    if (!(v[i] > 0.0) || !std::isfinite(v[i])) return false;
    sum += v[i];
  }
  return true;
}

pins_status Solver::prepare(const pins_config& cfg, const pins_problem& p, bool need_kcap) {
  err_.clear();
  int kind = kind_of(p.kind);
  if (kind < 0) { err_ = "unknown cost kind"; return PINS_ERR_INVALID_ARG; }
  if (p.m < 1 || p.n < 1) { err_ = "m and n must be >= 1"; return PINS_ERR_INVALID_ARG; }
  if ((long long)p.m * p.n > (1LL << 40)) { err_ = "m*n too large"; return PINS_ERR_INVALID_ARG; }
  if (!(cfg.eta > 0.0) || !std::isfinite(cfg.eta)) { err_ = "eta must be > 0"; return PINS_ERR_INVALID_ARG; }
  if (!p.a || !p.b) { err_ = "a and b are required"; return PINS_ERR_INVALID_ARG; }
  if (kind == COST_DENSE && !p.C) { err_ = "dense cost requires C"; return PINS_ERR_INVALID_ARG; }
  if (kind == COST_POINTS && (!p.x || !p.y || p.d < 1 || p.d > 4)) {
    err_ = "points cost requires x, y and 1 <= d <= 4"; return PINS_ERR_INVALID_ARG;
  }
  if (kind == COST_GRID && (p.grid_s1 < 1 || p.grid_s2 < 1 || p.grid_s1 * p.grid_s2 != p.m ||
                            p.m != p.n)) {
    err_ = "grid cost requires m = n = grid_s1 * grid_s2"; return PINS_ERR_INVALID_ARG;
  }
  if (kind != COST_DENSE && !(p.cost_scale > 0.0 && std::isfinite(p.cost_scale))) {
    err_ = "cost_scale must be > 0"; return PINS_ERR_INVALID_ARG;
  }
  if (kind == COST_GRID && (double)(p.grid_s1 - 1) * (p.grid_s1 - 1) +
                               (double)(p.grid_s2 - 1) * (p.grid_s2 - 1) > 16777216.0) {
    err_ = "grid too large for exact FP32 squared distances"; return PINS_ERR_INVALID_ARG;
  }
  // marginals: positive, finite, each summing to 1 (Eq. ot)
  std::vector<double> ha, hb;
  const double* pa = p.a;
  const double* pb = p.b;
  if (p.on_device) {
    ha.resize(p.m); hb.resize(p.n);
    cudaMemcpy(ha.data(), p.a, sizeof(double) * p.m, cudaMemcpyDeviceToHost);
    cudaMemcpy(hb.data(), p.b, sizeof(double) * p.n, cudaMemcpyDeviceToHost);
    if (check("reading a, b") != PINS_OK) return PINS_ERR_INVALID_ARG;
    pa = ha.data(); pb = hb.data();
  }
  double sa, sb;
  if (!vec_ok(pa, p.m, sa) || !vec_ok(pb, p.n, sb)) {
    err_ = "a and b must be finite and > 0"; return PINS_ERR_INVALID_ARG;
  }
  if (std::fabs(sa - 1.0) > 1e-9 || std::fabs(sb - 1.0) > 1e-9) {
    err_ = "a and b must each sum to 1 (within 1e-9)"; return PINS_ERR_INVALID_ARG;
  }
  if (!p.on_device && kind == COST_DENSE) {
    size_t mn = (size_t)p.m * p.n;
    if (p.kind == PINS_COST_DENSE_F64) {
      const double* C = (const double*)p.C;
      for (size_t e = 0; e < mn; ++e) if (!std::isfinite(C[e])) { err_ = "C has a non-finite entry"; return PINS_ERR_INVALID_ARG; }
    } else {
      const float* C = (const float*)p.C;
      for (size_t e = 0; e < mn; ++e) if (!std::isfinite(C[e])) { err_ = "C has a non-finite entry"; return PINS_ERR_INVALID_ARG; }
    }
  }
  mixed_ = (cfg.prec == PINS_PREC_MIXED);
  ps_ = mixed_ ? passes_mixed(kind) : passes_f64(kind);
  m_ = p.m; n_ = p.n; eta_ = cfg.eta;
  geom_ = make_geom(m_, n_);
  // the kept entries of a Newton step, and the certificate's support: the
  // 2(m + n - 1) largest entries (reading R9 (ii))
  int kcap = need_kcap ? solve_kcap(cfg, m_, n_)
                       : (int)std::min<long long>((long long)m_ * n_, 2LL * (m_ + n_ - 1));
  int t1cap = std::max(cfg.T1, 1);
  pins_status s = ensure(m_, n_, kcap, t1cap, p.kind, mixed_, !p.on_device, p.d);
  if (s != PINS_OK) return s;
  return upload(p);
}

pins_status Solver::upload(const pins_problem& p) {
  const bool host = !p.on_device;
  const size_t mn = (size_t)p.m * p.n;
  const cudaMemcpyKind H2D = cudaMemcpyHostToDevice;
  if (host) {
    cudaMemcpyAsync(ws_.a, p.a, sizeof(double) * p.m, H2D, stream_);
    cudaMemcpyAsync(ws_.b, p.b, sizeof(double) * p.n, H2D, stream_);
    a_ = ws_.a; b_ = ws_.b;
  } else {
    a_ = p.a; b_ = p.b;
  }
  cost_ = CostArgs{};
  cost_.m = p.m; cost_.n = p.n; cost_.d = p.d < 1 ? 1 : p.d;
  cost_.kind = kind_of(p.kind);
  cost_.scale = p.cost_scale;
  cost_.s2 = p.grid_s2;
  switch (p.kind) {
    case PINS_COST_DENSE_F64:
      if (!mixed_) {
        if (host) { cudaMemcpyAsync(ws_.C64, p.C, sizeof(double) * mn, H2D, stream_); cost_.C64 = ws_.C64; }
        else cost_.C64 = (const double*)p.C;
      } else {
        const double* src = (const double*)p.C;
        if (host) { cudaMemcpyAsync(ws_.C64, p.C, sizeof(double) * mn, H2D, stream_); src = ws_.C64; }
        launch_d2f(src, ws_.C32, mn, stream_); ++launches_;
        cost_.C32 = ws_.C32;
      }
      break;
    case PINS_COST_DENSE_F32:
      if (!mixed_) {
        const float* src = (const float*)p.C;
        if (host) { cudaMemcpyAsync(ws_.C32, p.C, sizeof(float) * mn, H2D, stream_); src = ws_.C32; }
        launch_f2d(src, ws_.C64, mn, stream_); ++launches_;
        cost_.C64 = ws_.C64;
      } else {
        if (host) { cudaMemcpyAsync(ws_.C32, p.C, sizeof(float) * mn, H2D, stream_); cost_.C32 = ws_.C32; }
        else cost_.C32 = (const float*)p.C;
      }
      break;
    case PINS_COST_POINTS_SQEUCLID: {
      const double* x = p.x;
      const double* y = p.y;
      if (host) {
        cudaMemcpyAsync(ws_.x, p.x, sizeof(double) * p.m * cost_.d, H2D, stream_);
        cudaMemcpyAsync(ws_.y, p.y, sizeof(double) * p.n * cost_.d, H2D, stream_);
        x = ws_.x; y = ws_.y;
      }
      cost_.x = x; cost_.y = y;
      if (mixed_) {
        launch_d2f(x, ws_.xf, (size_t)p.m * cost_.d, stream_);
        launch_d2f(y, ws_.yf, (size_t)p.n * cost_.d, stream_);
        launches_ += 2;
        cost_.xf = ws_.xf; cost_.yf = ws_.yf;
      }
      break;
    }
    case PINS_COST_GRID_SQEUCLID:
      if (mixed_) { launch_log_ab(a_, b_, p.m, p.n, ws_.lab, stream_); ++launches_; }
      break;
  }
  return check("upload");
}

PassArgs Solver::args(double s, const double* F, const double* G) {
  PassArgs a{};
  a.cost = cost_;
  a.m = m_; a.n = n_;
  a.eta = eta_; a.inv_eta = 1.0 / eta_; a.s = s;
  a.kappa = s / eta_;
  double craw = (cost_.kind == COST_DENSE) ? 1.0 : cost_.scale;
  double kd = a.kappa * craw;
  a.kappa_dd.hi = (float)kd;
  a.kappa_dd.lo = (float)(kd - (double)a.kappa_dd.hi);
  a.cscale = craw;
  a.F = F; a.G = G;
  a.A64 = ws_.A64; a.B64 = ws_.B64;
  a.Add = ws_.Add; a.Bdd = ws_.Bdd;
  const double L2E = 1.4426950408889634074;
  const double le = L2E / eta_, sl = s * L2E;
  a.l2e_eta = make_float2((float)le, (float)(le - (double)(float)le));
  a.s_l2e = make_float2((float)sl, (float)(sl - (double)(float)sl));
  const double k2 = kd * L2E;
  a.kappa2_dd.hi = (float)k2;
  a.kappa2_dd.lo = (float)(k2 - (double)a.kappa2_dd.hi);
  a.a = a_; a.b = b_;
  const bool lab = mixed_ && cost_.kind == COST_GRID;
  a.la = lab ? ws_.lab : nullptr;
  a.lb = lab ? ws_.lab + m_ : nullptr;
  a.exp_table = exp_table_;
  a.err = reinterpret_cast<int*>(ws_.scal + SC_FLAG);
  return a;
}

void Solver::prep(double s) {
  // (called with the solver's own F, G)
  prof_begin(PC_VEC);
  launch_prep(ws_.F, ws_.G, m_, n_, eta_, s, mixed_ ? nullptr : ws_.A64,
              mixed_ ? nullptr : ws_.B64, mixed_ ? ws_.Add : nullptr, mixed_ ? ws_.Bdd : nullptr,
              stream_);
  prof_end();
  ++launches_;
}

void Solver::sinkhorn_iter(double s, int t, bool with_res) {
  // the streamed mixed passes form their potentials from F, G themselves; Add/Bdd
  // are refreshed by the next prep() before any other pass.  Sizes whose row
  // segment or row block does not fit in shared memory use the tiled kernels,
  // which read Add/Bdd.
  const bool tiled = n_ > 32 * (PINS_ROW_SEG_SMEM_BYTES / 8) || m_ > 64 * (PINS_ROW_SEG_SMEM_BYTES / 8);
  auto refresh = [&]() {
    if (!mixed_ || tiled) prep(s);
  };
  refresh();
  PassArgs pa = args(s, ws_.F, ws_.G);
  prof_begin(PC_ROW_LSE);
  launches_ += ps_->row_lse(pa, geom_, ws_.mws, ws_.F,
                            with_res ? ws_.scal + SC_ROWRES + t : nullptr, stream_);
  prof_end();
  refresh();
  prof_begin(PC_COL_LSE);
  launches_ += ps_->col_lse(pa, geom_, ws_.mws, ws_.G, stream_);
  prof_end();
}

void Solver::marg(double s, bool trial, double alpha) {
  PassArgs pa = args(s, ws_.F, ws_.G);
  prof_begin(trial ? PC_TRIAL : PC_MARG);
  if (trial) {
    const double sc = alpha / eta_;
    TrialArgs tr{ws_.Pt64, ws_.Qt64, ws_.dir,
                 make_float2((float)sc, (float)(sc - (double)(float)sc))};
    ps_->marg(pa, geom_, ws_.mws, &tr, ws_.rt, ws_.ct, ws_.scal + SC_TRIAL, stream_);
  } else {
    ps_->marg(pa, geom_, ws_.mws, nullptr, ws_.r, ws_.c, ws_.scal + SC_MARG, stream_);
  }
  prof_end();
  ++launches_;
}

pins_status Solver::sparsify(double s, int keep, double zmax, int* nnz_out, bool csc) {
  // window: 64 nats of z below the largest key (X~ ratio e^-64), widened or
  // refined by the select kernel until the threshold bin fits the candidates
  SparsifyState st{};
  double width;
  if (!mixed_) {
    st.kref = eta_ * zmax + 1e-9 * (1.0 + s + std::fabs(eta_ * zmax));
    width = 64.0 * eta_ / PINS_HIST_NB;
  } else {
    st.kref = zmax + 1e-3 * (1.0 + std::fabs(zmax));
    width = 64.0 / PINS_HIST_NB;
  }
  st.inv_width = 1.0 / width;
  st.kref_f = (float)st.kref;
  st.inv_width_f = (float)st.inv_width;
  st.lo = 0.0; st.lo_f = 0.0f; st.count_in = 0; st.level = 0; st.done = 0; st.need = 0;
  st.thr_bin = -1; st.cand_count = 0; st.overflow = 0; st.keep = keep;
  st.tau = 0.0; st.tau_idx = -1;
  cudaMemcpyAsync(ws_.st, &st, sizeof(st), cudaMemcpyHostToDevice, stream_);
  cudaMemsetAsync(ws_.sw.rowcnt, 0, sizeof(int) * m_, stream_);
  PassArgs pa = args(s, ws_.F, ws_.G);
  int blocks = std::min(std::max((m_ + 7) / 8, 1), sms_ * 8);
  SparsifyState* hs = reinterpret_cast<SparsifyState*>(h_scal_ + SC_STATE);
  for (int round = 0; round < 13; ++round) {
    prof_begin(PC_HIST);
    ps_->key_hist(pa, ws_.st, ws_.hist, blocks, stream_);
    prof_end();
    prof_begin(PC_SELECT);
    launch_key_select(ws_.st, ws_.hist, (long long)m_ * n_, stream_);
    prof_end();
    prof_begin(PC_COMPACT);
    ps_->key_compact(pa, ws_.st, ws_.cand_key, ws_.cand_idx, ws_.sw.rowcnt, blocks, stream_);
    prof_end();
    prof_begin(PC_SELECT);
    cudaError_t cse = launch_cand_select(ws_.st, ws_.cand_key, ws_.cand_idx, n_, ws_.sw.rowcnt, stream_);
    prof_end();
    if (cse !=
        cudaSuccess) {
      return check("sparsify select");
    }
    launches_ += 4;
    cudaMemcpyAsync(hs, ws_.st, sizeof(SparsifyState), cudaMemcpyDeviceToHost, stream_);
    pins_status e = sync("sparsify");
    if (e != PINS_OK) return e;
    if (hs->done) break;
  }
  if (!hs->done || hs->overflow) {
    err_ = "sparsify: threshold selection failed (more tied keys than the candidate buffer)";
    return PINS_ERR_CUDA;
  }
  prof_begin(PC_WRITE);
  launch_scan(ws_.sw.rowcnt, ws_.sw.indptr, m_, stream_);
  ps_->key_write(pa, ws_.st, ws_.sw.indptr, ws_.sw.indices, ws_.sw.data, blocks, stream_);
  prof_end();
  launches_ += 2;
  if (csc) {
    prof_begin(PC_CSC);
    build_csc_from_csr(ws_.sw.indptr, ws_.sw.indices, ws_.sw.data, m_, n_, keep, ws_.sw, stream_);
    prof_end();
    launches_ += 5;
  }
  *nnz_out = keep;
  return check("csr");
}

void Solver::sparsify_fast(double s, int keep, float tau_guess) {
  FastSelState* fs = reinterpret_cast<FastSelState*>(ws_.scal + SC_FAST);
  PassArgs pa = args(s, ws_.F, ws_.G);
  const int blocks = std::min(std::max((m_ + 7) / 8, 1), sms_ * 8);
  prof_begin(PC_COMPACT);
  ps_->fast_collect(pa, tau_guess, fs, ws_.fkey, ws_.fij, blocks, stream_);
  prof_end();
  prof_begin(PC_SELECT);
  launch_fast_select(fs, ws_.fkey, ws_.fij, keep, stream_);
  prof_end();
  prof_begin(PC_WRITE);
  build_sparse_from_candidates(fs, ws_.fkey, ws_.fij, m_, n_, keep, ws_.sw, stream_);
  prof_end();
  launches_ += 7;
}

pins_status Solver::certificate(double s, double zmax) {
  // support-tree dual (reading R9 (ii)): the 2(m + n - 1) largest entries, a
  // maximum-weight spanning forest, potentials tight on its edges.  Where the
  // selection cannot resolve its threshold (more tied keys than the candidate
  // buffer), the tree dual is the entropic one and the bound is unchanged.
  const int ksup = (int)std::min<long long>((long long)m_ * n_, 2LL * (m_ + n_ - 1));
  int nnz = 0;
  prep(s);
  const std::string err_keep = err_;
  const bool have_tree = ksup <= ws_.kcap && sparsify(s, ksup, zmax, &nnz, false) == PINS_OK;
  launch_cert_pre(a_, ws_.r, ws_.F, m_, s, eta_, ws_.xs, ws_.u, stream_);
  ++launches_;
  PassArgs pa = args(s, ws_.F, ws_.G);
  prof_begin(PC_CERT);
  if (have_tree) {
    ps_->tree_duals(pa, ws_.sw.indptr, ws_.sw.indices, ksup, ws_.tw, ws_.uT,
                    reinterpret_cast<int*>(ws_.scal + SC_FLAG), stream_);
  } else {
    err_ = err_keep;
    cudaGetLastError();
    cudaMemcpyAsync(ws_.uT, ws_.u, sizeof(double) * m_, cudaMemcpyDeviceToDevice, stream_);
  }
  CertArgs ca{ws_.xs, ws_.ys, ws_.u, ws_.v, ws_.ec, ws_.c1, ws_.v, ws_.rr, ws_.cr, ws_.cp,
              ws_.tc, ws_.u2, ws_.uT, ws_.vT, ws_.vT, ws_.u2T};
  ps_->cert(pa, geom_, ws_.mws, ca, true, stream_);
  launch_cert_mid(b_, ws_.c1, n_, ws_.ys, ws_.ec, stream_);
  ps_->cert(pa, geom_, ws_.mws, ca, false, stream_);
  launch_cert_final(a_, b_, ws_.rr, ws_.cr, ws_.cp, ws_.tc, ws_.u2, ws_.v, ws_.u2T, ws_.vT, m_, n_,
                    ws_.scal + SC_CERT, ws_.scal + SC_CERT2, stream_);
  prof_end();
  launches_ += 5;
  return check("certificate");
}

pins_status Solver::solve(const pins_config& cfg, const pins_problem& p, pins_result& r) {
  auto t0 = std::chrono::steady_clock::now();
  long long launches0 = launches_;
  double* keepF = r.F_out;
  double* keepG = r.G_out;
  std::memset(&r, 0, sizeof(r));
  r.F_out = keepF; r.G_out = keepG;
  pins_status stt = prepare(cfg, p, true);
  if (stt != PINS_OK) { r.status = stt; return stt; }
  const int m = m_, n = n_;
  const int keep = (int)std::min<long long>((long long)m * n,
      std::max(1LL, (long long)llround(cfg.sparsify_gamma * (m + n - 1))));
  const int max_cg = std::max(1, std::min(cfg.max_cg, m + n));
  const double tol = cfg.tol_marg;
  const int check_every = std::max(1, cfg.sinkhorn_check_every);
  const int gap_every = std::max(1, cfg.gap_every);
  // state: F = G = Phi = Psi = 0 (readings R1); ab = (a; b)
  cudaMemsetAsync(ws_.F, 0, sizeof(double) * m, stream_);
  cudaMemsetAsync(ws_.G, 0, sizeof(double) * n, stream_);
  cudaMemsetAsync(ws_.Phi, 0, sizeof(double) * m, stream_);
  cudaMemsetAsync(ws_.Psi, 0, sizeof(double) * n, stream_);
  cudaMemcpyAsync(ws_.ab, a_, sizeof(double) * m, cudaMemcpyDeviceToDevice, stream_);
  cudaMemcpyAsync(ws_.ab + m, b_, sizeof(double) * n, cudaMemcpyDeviceToDevice, stream_);
  cudaMemsetAsync(ws_.scal + SC_FAST, 0, sizeof(FastSelState), stream_);
  // error flags of the kernels (CG index check, bulk-copy waits); any bit is fatal
  cudaMemsetAsync(ws_.scal + SC_FLAG, 0, sizeof(double), stream_);
  // one-pass selection between the Newton steps of an outer iteration (mixed path)
  const bool fast_path = mixed_ && cfg.sparsify_one_pass != 0 && ps_->fast_collect != nullptr &&
                         2 * keep <= PINS_FAST_CAP;
  float fast_margin = 1.0f;
  int outer = 0;
  bool stop = false, cert_current = false;
  double res = INFINITY, zmax = 0.0;
  double cert[4] = {0, 0, 0, 0};
  for (int k = 0; k < cfg.K && !stop; ++k) {
    const double s = (double)(k + 1);
    cert_current = false;
    // ---- Sinkhorn warm-up (readings R3, R4) ----
    // Blocks of check_every iterations (the residual of the block's last row
    // half-step decides the early exit).  Unprofiled solves launch a full block
    // as one CUDA graph, captured once per outer iteration (s is fixed within it).
    int t = 0;
    cudaGraphExec_t gexec = nullptr;
    long long glaunch = 0;                      // kernels in one graph launch
    bool use_graph = !profile_ && check_every >= 2;
    while (t < cfg.T1) {
      const int blk = std::min(check_every, cfg.T1 - t);
      bool launched = false;
      if (use_graph && blk == check_every) {
        if (!gexec) {
          cudaGraph_t graph = nullptr;
          const long long l0 = launches_;
          if (cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            for (int q = 0; q < blk; ++q) sinkhorn_iter(s, q, q == blk - 1);
            if (cudaStreamEndCapture(stream_, &graph) != cudaSuccess ||
                cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess)
              gexec = nullptr;
            if (graph) cudaGraphDestroy(graph);
          }
          glaunch = launches_ - l0;
          launches_ = l0;
          if (!gexec) { cudaGetLastError(); use_graph = false; }
        }
        if (gexec && cudaGraphLaunch(gexec, stream_) == cudaSuccess) {
          launches_ += glaunch;
          launched = true;
        }
      }
      if (!launched)
        for (int q = 0; q < blk; ++q) sinkhorn_iter(s, q, blk == check_every && q == blk - 1);
      t += blk;
      if (blk == check_every) {
        cudaMemcpyAsync(h_scal_ + SC_ROWRES + blk - 1, ws_.scal + SC_ROWRES + blk - 1,
                        sizeof(double), cudaMemcpyDeviceToHost, stream_);
        if ((stt = sync("warm-up")) != PINS_OK) {
          if (gexec) cudaGraphExecDestroy(gexec);
          r.status = stt;
          return stt;
        }
        if (h_scal_[SC_ROWRES + blk - 1] <= tol) break;
      }
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    r.sinkhorn_iters += t;
    // ---- sparse Newton (Alg. 2 second loop) ----
    prep(s);
    marg(s, false);
    cudaMemcpyAsync(h_scal_ + SC_MARG, ws_.scal + SC_MARG, 4 * sizeof(double),
                    cudaMemcpyDeviceToHost, stream_);
    if ((stt = sync("gradient")) != PINS_OK) { r.status = stt; return stt; }
    res = h_scal_[SC_MARG + 0];
    zmax = h_scal_[SC_MARG + 2];
    int steps = 0;
    bool fast_ok = false;      // this outer iteration has a CSR/CSC and an exact threshold
    float tau_prev = 0.f;
    while (steps < cfg.T2) {
      if (!(res > tol)) break;
      int nnz = 0;
      const bool fast = fast_path && fast_ok;
      if (fast) {
        // candidates above the previous threshold minus a margin; a failed
        // selection leaves the previous CSR/CSC and is redone below
        sparsify_fast(s, keep, tau_prev - fast_margin);
      } else {
        if ((stt = sparsify(s, keep, zmax, &nnz)) != PINS_OK) { r.status = stt; return stt; }
        tau_prev = (float)reinterpret_cast<const SparsifyState*>(h_scal_ + SC_STATE)->tau;
        fast_ok = fast_path;
      }
      // M d = grad with grad = (a - r; b - c); also <grad, d> and <ab, d> for the line search
      cudaError_t ce = run_cg(mixed_, m, n, eta_, ws_.r, ws_.c, ws_.sw.indptr, ws_.sw.indices,
                              ws_.sw.data, keep, nullptr, ws_.dir, cfg.cg_rtol, max_cg,
                              ws_.scal + SC_CG, ws_.ab, ws_.scal + SC_DOTS);
      if (ce != cudaSuccess) { err_ = std::string("cg launch: ") + cudaGetErrorString(ce); r.status = PINS_ERR_CUDA; return PINS_ERR_CUDA; }
      bool accepted = false, redo = false;
      double alpha = 1.0;
      int q = 0;
      for (; q <= cfg.max_backtrack; ++q) {
        if (!mixed_) {   // the mixed trial pass forms alpha d / eta itself
          launch_trial_prep(ws_.dir, m, n, alpha / eta_, ws_.Pt64, ws_.Qt64, nullptr, nullptr,
                            stream_);
          ++launches_;
        }
        marg(s, true, alpha);
        // trial scalars, dot products, CG info, the CG index-check flag and the
        // one-pass selection state in one copy
        cudaMemcpyAsync(h_scal_ + SC_TRIAL, ws_.scal + SC_TRIAL,
                        (SC_FAST + 4 - SC_TRIAL) * sizeof(double),
                        cudaMemcpyDeviceToHost, stream_);
        if ((stt = sync("line search")) != PINS_OK) { r.status = stt; return stt; }
        if (q == 0 && fast) {
          FastSelState f;
          std::memcpy(&f, h_scal_ + SC_FAST, sizeof(f));
          if (!f.fail && hooks_ && hooks_->select_fail.load() > 0 &&
              hooks_->select_fail.fetch_sub(1) > 0)
            f.fail = 2;
          if (f.fail) {
            // too few (1) or too many (2) candidates: widen or narrow the margin;
            // too many ties (3) or inconsistent counts: the histogram path
            if (f.fail == 1) fast_margin = std::min(64.0f, 2.0f * fast_margin);
            else if (f.fail == 2) fast_margin = std::max(1e-3f, 0.5f * fast_margin);
            redo = true;
            break;
          }
          tau_prev = f.tau;
          if (f.ncand > 3u * (unsigned)keep) fast_margin = std::max(1e-3f, 0.7f * fast_margin);
          else if (f.ncand < (unsigned)keep + keep / 4) fast_margin = std::min(64.0f, 1.4f * fast_margin);
        }
        if (q == 0) {
          r.cg_iters += (int)h_scal_[SC_CG];
          int flag = 0;
          std::memcpy(&flag, h_scal_ + SC_FLAG, sizeof(int));
          if (hooks_ && hooks_->kernel_error.load() > 0 && hooks_->kernel_error.fetch_sub(1) > 0)
            flag |= 64;
          if (flag) {
            err_ = std::string((flag & 64) ? "kernel error flag (injected by the test hook)"
                               : (flag & 16) ? "a bulk-copy wait gave up in a Sinkhorn pass"
                               : (flag & 128) ? "cg: a bulk-copy wait gave up"
                               : (flag & 32) ? "certificate: the spanning-forest build did not settle"
                                             : "cg: an index outside the cluster's slices was skipped") +
                   " (flag " + std::to_string(flag) + ")";
            r.status = PINS_ERR_CUDA;
            return PINS_ERR_CUDA;
          }
        }
        const double gtd = h_scal_[SC_DOTS + 0];
        const double adot = h_scal_[SC_DOTS + 1];
        const double dsum = h_scal_[SC_TRIAL + 3];
        // the trial pass's d term: sum X~ expm1(t) (FP64) or sum X~ (expm1(t) - t) (mixed)
        const double dP = mixed_ ? alpha * gtd - eta_ * dsum : alpha * adot - eta_ * dsum;
        if (std::isfinite(dP) && dP >= cfg.armijo_c1 * alpha * gtd) { accepted = true; break; }
        alpha *= cfg.armijo_beta;
      }
      if (redo) { fast_ok = false; continue; }   // same step again, histogram path
      r.ls_trials += std::min(q + 1, cfg.max_backtrack + 1);
      ++steps;
      if (accepted) {
        prof_begin(PC_VEC);
        launch_axpy_prep(ws_.F, ws_.G, ws_.dir, m, n, alpha, eta_, s, mixed_ ? nullptr : ws_.A64,
                         mixed_ ? nullptr : ws_.B64, mixed_ ? ws_.Add : nullptr,
                         mixed_ ? ws_.Bdd : nullptr, stream_);
        prof_end();
        ++launches_;
        std::swap(ws_.r, ws_.rt);
        std::swap(ws_.c, ws_.ct);
        res = h_scal_[SC_TRIAL + 0];
        zmax = h_scal_[SC_TRIAL + 2];
      } else {
        ++r.ls_failures;
        sinkhorn_iter(s, 0, false);
        prep(s);
        marg(s, false);
        cudaMemcpyAsync(h_scal_ + SC_MARG, ws_.scal + SC_MARG, 4 * sizeof(double),
                        cudaMemcpyDeviceToHost, stream_);
        if ((stt = sync("fallback")) != PINS_OK) { r.status = stt; return stt; }
        res = h_scal_[SC_MARG + 0];
        zmax = h_scal_[SC_MARG + 2];
      }
    }
    r.newton_iters += steps;
    outer = k + 1;
    // ---- outer stop (reading R9) ----
    if (cfg.tol_gap > 0.0 && (outer % gap_every == 0 || outer == cfg.K)) {
      if ((stt = certificate(s, zmax)) != PINS_OK) { r.status = stt; return stt; }
      cudaMemcpyAsync(cert, ws_.scal + SC_CERT, 4 * sizeof(double), cudaMemcpyDeviceToHost, stream_);
      if ((stt = sync("certificate")) != PINS_OK) { r.status = stt; return stt; }
      cert_current = true;
      if (cert[3] <= cfg.tol_gap) stop = true;
    }
    if (!stop && outer < cfg.K) {     // X^{k+1} becomes the next prox centre (R2)
      launch_outer(ws_.F, ws_.G, ws_.Phi, ws_.Psi, m, n, stream_);
      ++launches_;
    }
  }
  const double s_final = (double)outer;
  if (!cert_current) {
    if ((stt = certificate(s_final, zmax)) != PINS_OK) { r.status = stt; return stt; }
    cudaMemcpyAsync(cert, ws_.scal + SC_CERT, 4 * sizeof(double), cudaMemcpyDeviceToHost, stream_);
  }
  if (r.F_out) cudaMemcpyAsync(r.F_out, ws_.F, sizeof(double) * m, cudaMemcpyDeviceToHost, stream_);
  if (r.G_out) cudaMemcpyAsync(r.G_out, ws_.G, sizeof(double) * n, cudaMemcpyDeviceToHost, stream_);
  if ((stt = sync("result")) != PINS_OK) { r.status = stt; return stt; }
  r.cost = cert[0]; r.cost_ub = cert[1]; r.dual_lb = cert[2]; r.rel_gap = cert[3];
  r.marg_resid_l1 = res;
  r.s = s_final;
  r.outer_iters = outer;
  r.gpu_launches = (int)(launches_ - launches0);
  r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  bool converged = (cfg.tol_gap > 0.0) ? stop : (res <= tol);
  r.status = converged ? PINS_OK : PINS_ERR_NOT_CONVERGED;
  return r.status;
}

// ------------------------------------------------------------------------- //
// step-level entry points
// ------------------------------------------------------------------------- //
pins_status Solver::step_sinkhorn(const pins_config& cfg, const pins_problem& p, double s,
                                  int iters, double* F, double* G, double* row_res) {
  pins_config c2 = cfg;
  c2.T1 = std::max(cfg.T1, iters);
  pins_status st = prepare(c2, p, false);
  if (st != PINS_OK) return st;
  cudaMemcpyAsync(ws_.F, F, sizeof(double) * m_, cudaMemcpyDeviceToDevice, stream_);
  cudaMemcpyAsync(ws_.G, G, sizeof(double) * n_, cudaMemcpyDeviceToDevice, stream_);
  for (int t = 0; t < iters; ++t) sinkhorn_iter(s, t);
  cudaMemcpyAsync(F, ws_.F, sizeof(double) * m_, cudaMemcpyDeviceToDevice, stream_);
  cudaMemcpyAsync(G, ws_.G, sizeof(double) * n_, cudaMemcpyDeviceToDevice, stream_);
  if (row_res && iters > 0)
    cudaMemcpyAsync(row_res, ws_.scal + SC_ROWRES, sizeof(double) * iters,
                    cudaMemcpyDeviceToDevice, stream_);
  return sync("step_sinkhorn");
}

pins_status Solver::step_marginals(const pins_config& cfg, const pins_problem& p, double s,
                                   const double* F, const double* G, double* r, double* c,
                                   double* out3) {
  pins_status st = prepare(cfg, p, false);
  if (st != PINS_OK) return st;
  cudaMemcpyAsync(ws_.F, F, sizeof(double) * m_, cudaMemcpyDeviceToDevice, stream_);
  cudaMemcpyAsync(ws_.G, G, sizeof(double) * n_, cudaMemcpyDeviceToDevice, stream_);
  prep(s);
  marg(s, false);
  cudaMemcpyAsync(r, ws_.r, sizeof(double) * m_, cudaMemcpyDeviceToDevice, stream_);
  cudaMemcpyAsync(c, ws_.c, sizeof(double) * n_, cudaMemcpyDeviceToDevice, stream_);
  cudaMemcpyAsync(h_scal_ + SC_MARG, ws_.scal + SC_MARG, 4 * sizeof(double),
                  cudaMemcpyDeviceToHost, stream_);
  if ((st = sync("step_marginals")) != PINS_OK) return st;
  double o[3] = {h_scal_[SC_MARG], h_scal_[SC_MARG + 1], eta_ * h_scal_[SC_MARG + 2]};
  cudaMemcpyAsync(out3, o, sizeof(o), cudaMemcpyHostToDevice, stream_);
  return sync("step_marginals out");
}

pins_status Solver::step_sparsify(const pins_config& cfg, const pins_problem& p, double s,
                                  const double* F, const double* G, int keep, int* indptr,
                                  int* indices, double* data) {
  if (keep < 1 || (long long)keep > (long long)p.m * p.n) { err_ = "keep out of range"; return PINS_ERR_INVALID_ARG; }
  pins_config c2 = cfg;
  c2.sparsify_gamma = 1.0;
  pins_status st = prepare(c2, p, false);
  if (st != PINS_OK) return st;
  // the workspace must hold `keep` entries
  if ((st = ensure(m_, n_, keep, std::max(cfg.T1, 1), p.kind, mixed_, !p.on_device, p.d)) != PINS_OK) return st;
  if ((st = upload(p)) != PINS_OK) return st;
  cudaMemcpyAsync(ws_.F, F, sizeof(double) * m_, cudaMemcpyDeviceToDevice, stream_);
  cudaMemcpyAsync(ws_.G, G, sizeof(double) * n_, cudaMemcpyDeviceToDevice, stream_);
  prep(s);
  marg(s, false);
  cudaMemcpyAsync(h_scal_ + SC_MARG, ws_.scal + SC_MARG, 4 * sizeof(double),
                  cudaMemcpyDeviceToHost, stream_);
  if ((st = sync("step_sparsify marg")) != PINS_OK) return st;
  int nnz = 0;
  if ((st = sparsify(s, keep, h_scal_[SC_MARG + 2], &nnz)) != PINS_OK) return st;
  cudaMemcpyAsync(indptr, ws_.sw.indptr, sizeof(int) * (m_ + 1), cudaMemcpyDeviceToDevice, stream_);
  cudaMemcpyAsync(indices, ws_.sw.indices, sizeof(int) * keep, cudaMemcpyDeviceToDevice, stream_);
  cudaMemcpyAsync(data, ws_.sw.data, sizeof(double) * keep, cudaMemcpyDeviceToDevice, stream_);
  return sync("step_sparsify");
}

cudaError_t Solver::run_cg(bool mixed, int m, int n, double eta, const double* r,
                           const double* c, const int* indptr, const int* indices,
                           const double* data, int nnz, const double* rhs, double* d,
                           double rtol, int max_iter, double* info, const double* ab,
                           double* dots) {
  prof_begin(PC_CG);
  if (mixed) {
    // the double-float kernel forms rhs = ab - (r; c) itself when rhs is NULL and
    // writes the two inner products of the line search
    bool used = false;
    cudaError_t ce = launch_pcg_dd(m, n, eta, r, c, indptr, indices, data, ws_.sw.colptr,
                                   ws_.sw.rowidx, ws_.sw.cdata, rhs, d, ab, dots, ws_.ent_tgt,
                                   ws_.ent_val, ws_.ent_row, ws_.cg_u, nnz, rtol, max_iter, info,
                                   reinterpret_cast<int*>(ws_.scal + SC_FLAG), stream_, &used);
    if (used) { prof_end(); ++launches_; return ce; }
  }
  if (!rhs) {
    launch_grad(a_, b_, r, c, m, n, ws_.grad, stream_);
    rhs = ws_.grad;
    ++launches_;
  }
  cudaError_t ce = launch_pcg(m, n, eta, r, c, indptr, indices, data, ws_.sw.colptr,
                              ws_.sw.rowidx, ws_.sw.cdata, rhs, d, ws_.cg_res, ws_.cg_p, ws_.cg_q,
                              ws_.cg_part, rtol, max_iter, info,
                              reinterpret_cast<int*>(ws_.scal + SC_FLAG), sms_, stream_);
  prof_end();
  ++launches_;
  if (dots) {
    launch_dot2(rhs, d, ab, d, m + n, dots, stream_);
    ++launches_;
  }
  return ce;
}

pins_status Solver::step_cg(int m, int n, double eta, const double* r, const double* c,
                            const int* indptr, const int* indices, const double* data, int nnz,
                            const double* rhs, double* d, double rtol, int max_iter,
                            double* info, bool mixed) {
  err_.clear();
  if (m < 1 || n < 1 || nnz < 0 || !(eta > 0.0) || max_iter < 0) { err_ = "bad CG arguments"; return PINS_ERR_INVALID_ARG; }
  pins_status st = ensure(m, n, std::max(nnz, 1), 1, PINS_COST_GRID_SQEUCLID, false, false, 1);
  if (st != PINS_OK) return st;
  build_csc_from_csr(indptr, indices, data, m, n, nnz, ws_.sw, stream_);
  cudaMemsetAsync(ws_.scal + SC_FLAG, 0, sizeof(double), stream_);   // index-check flag
  cudaError_t ce = run_cg(mixed, m, n, eta, r, c, indptr, indices, data, nnz, rhs, d, rtol,
                          max_iter, info, nullptr, nullptr);
  launches_ += 6;
  if (ce != cudaSuccess) { err_ = std::string("cg launch: ") + cudaGetErrorString(ce); return PINS_ERR_CUDA; }
  return sync("step_cg");
}

pins_status Solver::step_objective_increase(const pins_config& cfg, const pins_problem& p,
                                            double s, const double* F, const double* G,
                                            const double* df, const double* dg, double alpha,
                                            double* out) {
  pins_status st = prepare(cfg, p, false);
  if (st != PINS_OK) return st;
  cudaMemcpyAsync(ws_.F, F, sizeof(double) * m_, cudaMemcpyDeviceToDevice, stream_);
  cudaMemcpyAsync(ws_.G, G, sizeof(double) * n_, cudaMemcpyDeviceToDevice, stream_);
  cudaMemcpyAsync(ws_.dir, df, sizeof(double) * m_, cudaMemcpyDeviceToDevice, stream_);
  cudaMemcpyAsync(ws_.dir + m_, dg, sizeof(double) * n_, cudaMemcpyDeviceToDevice, stream_);
  cudaMemcpyAsync(ws_.ab, a_, sizeof(double) * m_, cudaMemcpyDeviceToDevice, stream_);
  cudaMemcpyAsync(ws_.ab + m_, b_, sizeof(double) * n_, cudaMemcpyDeviceToDevice, stream_);
  prep(s);
  if (mixed_) {
    // the mixed trial pass returns sum X~ (expm1(t) - t); the linear part is
    // alpha <grad, d> with grad = (a - r, b - c) at the current point
    marg(s, false);
    launch_grad(a_, b_, ws_.r, ws_.c, m_, n_, ws_.grad, stream_);
    launch_dot2(ws_.grad, ws_.dir, nullptr, nullptr, m_ + n_, ws_.scal + SC_DOTS, stream_);
    launches_ += 2;
  } else {
    launch_dot2(ws_.ab, ws_.dir, nullptr, nullptr, m_ + n_, ws_.scal + SC_DOTS, stream_);
    ++launches_;
  }
  if (!mixed_)
    launch_trial_prep(ws_.dir, m_, n_, alpha / eta_, ws_.Pt64, ws_.Qt64, nullptr, nullptr,
                      stream_);
  marg(s, true, alpha);
  ++launches_;
  cudaMemcpyAsync(h_scal_, ws_.scal, 16 * sizeof(double), cudaMemcpyDeviceToHost, stream_);
  if ((st = sync("step_objective_increase")) != PINS_OK) return st;
  double dP = alpha * h_scal_[SC_DOTS] - eta_ * h_scal_[SC_TRIAL + 3];
  if (!std::isfinite(dP)) dP = -INFINITY;
  cudaMemcpyAsync(out, &dP, sizeof(double), cudaMemcpyHostToDevice, stream_);
  return sync("step_objective_increase out");
}

pins_status Solver::step_certificate(const pins_config& cfg, const pins_problem& p, double s,
                                     const double* F, const double* G, double* out6) {
  pins_status st = prepare(cfg, p, false);
  if (st != PINS_OK) return st;
  cudaMemcpyAsync(ws_.F, F, sizeof(double) * m_, cudaMemcpyDeviceToDevice, stream_);
  cudaMemcpyAsync(ws_.G, G, sizeof(double) * n_, cudaMemcpyDeviceToDevice, stream_);
  prep(s);
  marg(s, false);
  cudaMemcpyAsync(h_scal_ + SC_MARG, ws_.scal + SC_MARG, 4 * sizeof(double),
                  cudaMemcpyDeviceToHost, stream_);
  if ((st = sync("step_certificate marg")) != PINS_OK) return st;
  if ((st = certificate(s, h_scal_[SC_MARG + 2])) != PINS_OK) return st;
  cudaMemcpyAsync(out6, ws_.scal + SC_CERT, 4 * sizeof(double), cudaMemcpyDeviceToDevice, stream_);
  cudaMemcpyAsync(out6 + 4, ws_.scal + SC_CERT2, 2 * sizeof(double), cudaMemcpyDeviceToDevice,
                  stream_);
  return sync("step_certificate");
}

}  // namespace pins
