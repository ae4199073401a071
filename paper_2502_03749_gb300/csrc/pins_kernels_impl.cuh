// Instantiates the pass kernels for one arithmetic policy and every cost kind.
// Included once per policy translation unit with PINS_POLICY and PINS_PASSES_FN set.
#include "pins_sparsify.cuh"
#include "pins_kernels.h"

namespace pins {
namespace {

template <int K> struct Launch {
  using P = PINS_POLICY<K>;
  static void row_lse(const PassArgs& p, const TileGeom& g, const MergeWS& ws, double* F_out,
                      double* out_res, cudaStream_t st) {
    k_row_lse<P><<<dim3(g.gx, g.gy), PINS_TPB, 0, st>>>(p, g, ws, F_out, out_res);
  }
  static void col_lse(const PassArgs& p, const TileGeom& g, const MergeWS& ws, double* G_out,
                      cudaStream_t st) {
    k_col_lse<P><<<dim3(g.gx, g.gy), PINS_TPB, 0, st>>>(p, g, ws, G_out);
  }
  static void marg(const PassArgs& p, const TileGeom& g, const MergeWS& ws, const TrialArgs* tr,
                   double* r, double* c, double* out4, cudaStream_t st) {
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
  static const PassSet* get() {
    static const PassSet ps = {P::MIXED, row_lse, col_lse, marg, cert, key_hist, key_compact,
                               key_write};
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
