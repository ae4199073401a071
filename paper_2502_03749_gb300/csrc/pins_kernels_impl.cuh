// Instantiates the pass kernels for one arithmetic policy and every cost kind.
// Included once per policy translation unit with PINS_POLICY and PINS_PASSES_FN set.
#include "pins_sparsify.cuh"
#include "pins_kernels.h"
#include <algorithm>

namespace pins {
namespace {

// function-local statics below are initialised once, thread-safely (the serving
// workers launch from several threads)
int sm_count() {
  static const int v = [] {
    int d = 0, x = 0;
    cudaGetDevice(&d);
    if (cudaDeviceGetAttribute(&x, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || x <= 0)
      x = 152;
    return x;
  }();
  return v;
}

#define PINS_ROW_SEG_SMEM PINS_ROW_SEG_SMEM_BYTES

template <int K> struct Launch {
  using P = PINS_POLICY<K>;
  // grid cost of the mixed policy: the separable two-stage half-step, when both
  // measures share the s1 x s2 grid and the stage buffers fit (T in rowpart0,
  // one residual slot per grid column in scal_row, a column of T in 48 KB of
  // shared memory)
  static bool grid_separable(const PassArgs& p, int& s1, int& s2) {
    s2 = p.cost.s2;
    s1 = s2 > 0 ? p.m / s2 : 0;
    return K == COST_GRID && P::MIXED && s2 > 0 && p.m == p.n && s1 * s2 == p.m &&
           s2 <= 8 * PINS_GY_MAX && s1 <= 6144;
  }
  static int row_lse(const PassArgs& p, const TileGeom& g, const MergeWS& ws, double* F_out,
                     double* out_res, cudaStream_t st) {
    int s1, s2;
    if (grid_separable(p, s1, s2)) {
      k_grid_lse1<true><<<s1, PINS_TPB, sizeof(float2) * s2, st>>>(p, s1, s2, ws.rowpart0);
      k_grid_lse2<true><<<s2, PINS_TPB, sizeof(float2) * s1, st>>>(p, s1, s2, ws.rowpart0, ws,
                                                                     F_out, out_res);
      return 2;
    }
    if constexpr (P::MIXED) {
      // column segments of ~1024 (at most g.gx of them: rowpart0 holds g.gx * m),
      // row groups for ~4 CTAs per SM (at most PINS_ROW_GROUPS counters)
      const int sx = std::max(1, std::min(g.gx, (p.n + 1023) / 1024));
      const int seg = (((p.n + sx - 1) / sx) + PINS_TC - 1) / PINS_TC * PINS_TC;
      // dense 1024-column segments stream through per-warp bulk-copy buffers
      // (2 x 4 KB per warp): 3 CTAs per SM then
      const bool bulk = P::MIXED && K == COST_DENSE && (p.n % 4) == 0 && seg == 1024 &&
                        (reinterpret_cast<uintptr_t>(p.cost.C32) % 16) == 0;
      const size_t smem = sizeof(float2) * (size_t)seg + (bulk ? 2u * 4096u * PINS_WARPS : 0u);
      if (smem <= PINS_ROW_SEG_SMEM) {
        static const cudaError_t configured = cudaFuncSetAttribute(
            k_row_lse_mx<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, PINS_ROW_SEG_SMEM);
        (void)configured;
        const int per_sm = bulk ? 3 : 4;
        const int gy = std::max(1, std::min({(per_sm * sm_count() + sx - 1) / sx, PINS_ROW_GROUPS,
                                             (p.m + PINS_WARPS - 1) / PINS_WARPS}));
        k_row_lse_mx<P><<<dim3(sx, gy), PINS_TPB, smem, st>>>(p, seg, ws, F_out, out_res);
        return 1;
      }
    }
    k_row_lse<P><<<dim3(g.gx, g.gy), PINS_TPB, 0, st>>>(p, g, ws, F_out, out_res);
    return 1;
  }
  static int col_lse(const PassArgs& p, const TileGeom& g, const MergeWS& ws, double* G_out,
                     cudaStream_t st) {
    int s1, s2;
    if (grid_separable(p, s1, s2)) {
      k_grid_lse1<false><<<s1, PINS_TPB, sizeof(float2) * s2, st>>>(p, s1, s2, ws.rowpart0);
      k_grid_lse2<false><<<s2, PINS_TPB, sizeof(float2) * s1, st>>>(p, s1, s2, ws.rowpart0, ws,
                                                                      G_out, nullptr);
      return 2;
    }
    if constexpr (P::MIXED) {
      // row blocks for ~4 CTAs per SM, at most g.gy (colpart0 holds g.gy * n), and
      // enough of them for a block's A_i to fit in shared memory
      const int rows_fit = PINS_ROW_SEG_SMEM / (int)sizeof(float2);
      const int gy = std::max(1, std::min({std::max((4 * sm_count() + g.gx - 1) / g.gx,
                                                    (p.m + rows_fit - 1) / rows_fit),
                                           g.gy, (p.m + PINS_WARPS - 1) / PINS_WARPS}));
      const int rb = (p.m + gy - 1) / gy;
      const size_t smem = sizeof(float2) * (size_t)rb;
      if (smem <= PINS_ROW_SEG_SMEM) {
        static const cudaError_t configured = cudaFuncSetAttribute(
            k_col_lse_mx<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, PINS_ROW_SEG_SMEM);
        (void)configured;
        k_col_lse_mx<P><<<dim3(g.gx, gy), PINS_TPB, smem, st>>>(p, rb, ws, G_out);
        return 1;
      }
    }
    k_col_lse<P><<<dim3(g.gx, g.gy), PINS_TPB, 0, st>>>(p, g, ws, G_out);
    return 1;
  }
  static void marg(const PassArgs& p, const TileGeom& g, const MergeWS& ws, const TrialArgs* tr,
                   double* r, double* c, double* out4, cudaStream_t st) {
    if constexpr (P::MIXED) {
      // column segments of PINS_MSEG (at most g.gx: rowpart holds g.gx * m), row
      // groups for one wave at 2 CTAs per SM (at most g.gy: colpart holds g.gy * n)
      const int sx = (p.n + PINS_MSEG - 1) / PINS_MSEG;
      if (sx <= g.gx) {
        static const bool configured = [] {
          cudaFuncSetAttribute(k_marg_mx<P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)PINS_MSEG_SMEM);
          cudaFuncSetAttribute(k_marg_mx<P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)PINS_MSEG_SMEM);
          return true;
        }();
        (void)configured;
        const int gy = std::max(1, std::min({(2 * sm_count() + sx - 1) / sx, g.gy,
                                             (p.m + PINS_WARPS - 1) / PINS_WARPS}));
        if (tr) {
          k_marg_mx<P, true><<<dim3(sx, gy), PINS_TPB, PINS_MSEG_SMEM, st>>>(p, ws, *tr, r, c, out4);
        } else {
          TrialArgs none{};
          k_marg_mx<P, false><<<dim3(sx, gy), PINS_TPB, PINS_MSEG_SMEM, st>>>(p, ws, none, r, c, out4);
        }
        return;
      }
    }
    if (tr) k_marg<P, true><<<dim3(g.gx, g.gy), PINS_TPB, 0, st>>>(p, g, ws, *tr, r, c, out4);
    else {
      TrialArgs none{};
      k_marg<P, false><<<dim3(g.gx, g.gy), PINS_TPB, 0, st>>>(p, g, ws, none, r, c, out4);
    }
  }
  static void cert(const PassArgs& p, const TileGeom& g, const MergeWS& ws, const CertArgs& ca,
                   bool colpass, cudaStream_t st) {
    if (colpass) k_cert<P, true><<<dim3(g.gx, g.gy), PINS_TPB, 0, st>>>(p, g, ws, ca);
    else k_cert<P, false><<<dim3(g.gx, g.gy), PINS_TPB, 0, st>>>(p, g, ws, ca);
  }
  static void key_hist(const PassArgs& p, const SparsifyState* s, unsigned int* hist, int blocks,
                       cudaStream_t st) {
    k_key_hist<P><<<blocks, PINS_TPB, 0, st>>>(p, s, hist);
  }
  static void key_compact(const PassArgs& p, SparsifyState* s, double* ck, long long* ci,
                          int* rowcnt, int blocks, cudaStream_t st) {
    k_key_compact<P><<<blocks, PINS_TPB, 0, st>>>(p, s, ck, ci, rowcnt);
  }
  static void key_write(const PassArgs& p, const SparsifyState* s, const int* indptr, int* indices,
                        double* data, int blocks, cudaStream_t st) {
    k_key_write<P><<<blocks, PINS_TPB, 0, st>>>(p, s, indptr, indices, data);
  }
  static void fast_collect(const PassArgs& p, float tau_guess, FastSelState* fs, float* ckey,
                           unsigned long long* cij, int blocks, cudaStream_t st) {
    if constexpr (P::MIXED)
      k_fast_collect<P><<<blocks, PINS_TPB, 0, st>>>(p, tau_guess, fs, ckey, cij);
  }
  static void tree_duals(const PassArgs& p, const int* indptr, const int* indices, int ne,
                         const TreeWS& tw, double* uT, int* err, cudaStream_t st) {
    k_tree_duals<P><<<1, PINS_TREE_TPB, 0, st>>>(p, indptr, indices, ne, tw, uT, err);
  }
  static const PassSet* get() {
    static const PassSet ps = {P::MIXED, row_lse, col_lse, marg, cert, key_hist, key_compact,
                               key_write, P::MIXED ? fast_collect : nullptr, tree_duals};
    return &ps;
  }
};

}  // namespace

const PassSet* PINS_PASSES_FN(int kind) {
  switch (kind) {
    case COST_DENSE: return Launch<COST_DENSE>::get();
    case COST_POINTS: return Launch<COST_POINTS>::get();
    case COST_GRID: return Launch<COST_GRID>::get();
    default: return nullptr;
  }
}

}  // namespace pins
