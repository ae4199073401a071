// pins_marginals_noalloc: the marginal pass (row and column sums of the plan)
// for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not wanted --
// inside a framework whose device memory is owned by its own pool allocator, in
// a real-time loop that must not hit the driver's allocator (whose calls can
// synchronise the device and take milliseconds), or in an embedding that
// pre-reserves all memory at start-up.  The regular step entry points take a
// pins_handle, whose workspace is allocated on first use; this one needs no
// handle and allocates nothing.
//
// How: every scratch buffer the pass needs (cross-block partials, arrival
// counters, the per-row/column exponent pieces, the 2^(q/1024) table of the
// mixed path) is carved from one file-scope static device array of
// PINS_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds until
// the process exits.  Host code cannot pass that array's name to a kernel (the
// name is a host-side stand-in), so the first call on each device looks up its
// device address with cudaGetSymbolAddress while that device is current, fills
// the table, and caches the address.  That first call also copies from the host,
// so make it before any stream capture.
//
// All calls on one device share that device's copy of the array: it keeps the
// last call's contents, and the counters that must start at zero are cleared by
// every call.  Two calls whose work overlaps on the same GPU (for example on two
// streams without ordering between them) race on the shared scratch and give
// wrong results: order them on one stream or synchronise between them.
#include <mutex>
#include <vector>
#include <cmath>
#include "../../include/pins.h"
#include "pins_kernels.h"
#include "pins_sparsify.cuh"

namespace pins {
namespace {

constexpr int kMaxDim = PINS_NOALLOC_MAX_DIM;
constexpr size_t kScratchBytes = PINS_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Layout {   // offsets (bytes) into the scratch array, sized for kMaxDim
  size_t rowpart0, colpart0, scal_row, scal_col, cnt_row, cnt_col, cnt_all;
  size_t A64, B64, Add, Bdd, xf, yf, table, out4, end;
};

Layout layout() {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) { off = (off + 255) & ~size_t(255); size_t o = off; off += bytes; return o; };
  L.rowpart0 = take(sizeof(double) * PINS_GX_MAX * kMaxDim);
  L.colpart0 = take(sizeof(double) * PINS_GY_MAX * kMaxDim);
  L.scal_row = take(sizeof(double) * 8 * PINS_GY_MAX);
  L.scal_col = take(sizeof(double) * (4 * PINS_GX_MAX * PINS_GY_MAX + PINS_GX_MAX));
  L.cnt_row = take(sizeof(unsigned int) * PINS_GY_MAX);
  L.cnt_col = take(sizeof(unsigned int) * PINS_GX_MAX);
  L.cnt_all = take(sizeof(unsigned int));
  L.A64 = take(sizeof(double) * kMaxDim);
  L.B64 = take(sizeof(double) * kMaxDim);
  L.Add = take(sizeof(float2) * kMaxDim);
  L.Bdd = take(sizeof(float2) * kMaxDim);
  L.xf = take(sizeof(float) * 4 * kMaxDim);
  L.yf = take(sizeof(float) * 4 * kMaxDim);
  L.table = take(sizeof(float2) * PINS_EXP_TABLE);
  L.out4 = take(sizeof(double) * 4);
  L.end = off;
  return L;
}

static_assert(PINS_NOALLOC_MAX_DIM <= 4096, "scratch sized for m, n <= 4096");

std::mutex g_mu;
std::vector<unsigned char*> g_base;   // per device: device address of the array

// once per device, with that device current
cudaError_t scratch_base(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if ((int)g_base.size() <= dev) g_base.resize(dev + 1, nullptr);
  if (!g_base[dev]) {
    const Layout L = layout();
    if (L.end > kScratchBytes) return cudaErrorInvalidValue;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    std::vector<float2> tab(PINS_EXP_TABLE);
    for (int q = 0; q < PINS_EXP_TABLE; ++q) {
      const double v = std::exp2((double)q / PINS_EXP_TABLE);
      const float hi = (float)v;
      tab[q] = make_float2(hi, (float)(v - (double)hi));
    }
    e = cudaMemcpy(static_cast<unsigned char*>(p) + L.table, tab.data(),
                   sizeof(float2) * tab.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    g_base[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_base[dev];
  return cudaSuccess;
}

__global__ void k_noalloc_out3(const double* s4, double eta, double* out3) {
  out3[0] = s4[0];
  out3[1] = s4[1];
  out3[2] = eta * s4[2];
}

}  // namespace
}  // namespace pins

extern "C" pins_status pins_marginals_noalloc(const pins_problem* p, double eta, int prec,
                                              double s, const double* F, const double* G,
                                              double* r, double* c, double* out3,
                                              void* cuda_stream) {
  using namespace pins;
  if (!p || !F || !G || !r || !c || !out3 || !p->on_device || !p->a || !p->b)
    return PINS_ERR_INVALID_ARG;
  if (p->m < 1 || p->n < 1 || p->m > kMaxDim || p->n > kMaxDim) return PINS_ERR_INVALID_ARG;
  if (!(eta > 0.0) || !std::isfinite(eta) || !std::isfinite(s)) return PINS_ERR_INVALID_ARG;
  if (prec != PINS_PREC_FP64 && prec != PINS_PREC_MIXED) return PINS_ERR_INVALID_ARG;
  const bool mixed = (prec == PINS_PREC_MIXED);
  int kind;
  switch (p->kind) {
    case PINS_COST_DENSE_F64: if (mixed || !p->C) return PINS_ERR_INVALID_ARG; kind = COST_DENSE; break;
    case PINS_COST_DENSE_F32: if (!mixed || !p->C) return PINS_ERR_INVALID_ARG; kind = COST_DENSE; break;
    case PINS_COST_POINTS_SQEUCLID:
      if (!p->x || !p->y || p->d < 1 || p->d > 4 || !(p->cost_scale > 0.0)) return PINS_ERR_INVALID_ARG;
      kind = COST_POINTS; break;
    case PINS_COST_GRID_SQEUCLID:
      if (p->grid_s1 < 1 || p->grid_s2 < 1 || p->grid_s1 * p->grid_s2 != p->m || p->m != p->n ||
          !(p->cost_scale > 0.0))
        return PINS_ERR_INVALID_ARG;
      kind = COST_GRID; break;
    default: return PINS_ERR_INVALID_ARG;
  }
  // an error already pending from unrelated work is left for its owner: only
  // an error that appears during this call is reported (and cleared)
  const cudaError_t pending = cudaPeekAtLastError();
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return PINS_ERR_CUDA; }
  unsigned char* base = nullptr;
  if (scratch_base(dev, &base) != cudaSuccess) { cudaGetLastError(); return PINS_ERR_CUDA; }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const Layout L = layout();
  const int m = p->m, n = p->n;
  MergeWS ws{};
  ws.cnt_row = reinterpret_cast<unsigned int*>(base + L.cnt_row);
  ws.cnt_col = reinterpret_cast<unsigned int*>(base + L.cnt_col);
  ws.cnt_all = reinterpret_cast<unsigned int*>(base + L.cnt_all);
  ws.rowpart0 = reinterpret_cast<double*>(base + L.rowpart0);
  ws.colpart0 = reinterpret_cast<double*>(base + L.colpart0);
  ws.scal_row = reinterpret_cast<double*>(base + L.scal_row);
  ws.scal_col = reinterpret_cast<double*>(base + L.scal_col);
  // the arrival counters must start at zero (the kernel leaves them at zero, but
  // an earlier call that failed midway may not have)
  cudaMemsetAsync(base + L.cnt_row, 0, L.A64 - L.cnt_row, st);

  CostArgs cost{};
  cost.kind = kind; cost.m = m; cost.n = n; cost.d = p->d < 1 ? 1 : p->d;
  cost.scale = p->cost_scale; cost.s2 = p->grid_s2;
  if (kind == COST_DENSE) {
    if (mixed) cost.C32 = (const float*)p->C; else cost.C64 = (const double*)p->C;
  } else if (kind == COST_POINTS) {
    cost.x = p->x; cost.y = p->y;
    if (mixed) {
      float* xf = reinterpret_cast<float*>(base + L.xf);
      float* yf = reinterpret_cast<float*>(base + L.yf);
      launch_d2f(p->x, xf, (size_t)m * cost.d, st);
      launch_d2f(p->y, yf, (size_t)n * cost.d, st);
      cost.xf = xf; cost.yf = yf;
    }
  }
  PassArgs pa{};
  pa.cost = cost;
  pa.m = m; pa.n = n;
  pa.eta = eta; pa.inv_eta = 1.0 / eta; pa.s = s;
  pa.kappa = s / eta;
  const double craw = (kind == COST_DENSE) ? 1.0 : p->cost_scale;
  const double kd = pa.kappa * craw;
  pa.kappa_dd.hi = (float)kd;
  pa.kappa_dd.lo = (float)(kd - (double)pa.kappa_dd.hi);
  pa.cscale = craw;
  pa.F = F; pa.G = G;
  pa.A64 = reinterpret_cast<double*>(base + L.A64);
  pa.B64 = reinterpret_cast<double*>(base + L.B64);
  pa.Add = reinterpret_cast<float2*>(base + L.Add);
  pa.Bdd = reinterpret_cast<float2*>(base + L.Bdd);
  pa.a = p->a; pa.b = p->b;
  pa.exp_table = reinterpret_cast<float2*>(base + L.table);
  launch_prep(F, G, m, n, eta, s, mixed ? nullptr : reinterpret_cast<double*>(base + L.A64),
              mixed ? nullptr : reinterpret_cast<double*>(base + L.B64),
              mixed ? reinterpret_cast<float2*>(base + L.Add) : nullptr,
              mixed ? reinterpret_cast<float2*>(base + L.Bdd) : nullptr, st);
  const PassSet* ps = mixed ? passes_mixed(kind) : passes_f64(kind);
  const TileGeom g = make_geom(m, n);
  double* out4 = reinterpret_cast<double*>(base + L.out4);
  ps->marg(pa, g, ws, nullptr, r, c, out4, st);
  k_noalloc_out3<<<1, 1, 0, st>>>(out4, eta, out3);
  if (pending == cudaSuccess && cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return PINS_ERR_CUDA;
  }
  return PINS_OK;
}
