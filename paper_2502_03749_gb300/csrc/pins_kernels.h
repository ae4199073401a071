// Internal interface between the host solver and the kernel translation units.
#pragma once
#include <cuda_runtime.h>
#include "pins_common.cuh"

namespace pins {

// shared memory of one row segment (row LSE) or row block (column LSE) of the
// streamed mixed Sinkhorn kernels
#define PINS_ROW_SEG_SMEM_BYTES (96 * 1024)

struct SparsifyState;
struct TrialArgs;
struct CertArgs;
struct TreeWS;

// One-pass selection used between Newton steps of one outer iteration on the
// mixed path: every entry whose key is at least tau_guess (the previous step's
// threshold minus a margin) is collected; the exact top-K is then selected from
// the candidates.  Lives in the solver's scalar block (4 doubles), so the host
// reads it together with the line-search scalars.
#define PINS_FAST_CAP 49152     // candidate capacity (keys staged in one CTA's shared memory)
#define PINS_FAST_TIES 2048     // entries tied at the threshold key that can be ordered
struct FastSelState {
  unsigned int count;         // candidates found by the collect pass (may exceed the capacity)
  unsigned int ncand;         // candidates used by the select pass (0 on failure)
  int fail;                   // 1: fewer than K candidates, 2: too many, 3: too many ties
  int pad;
  float tau;                  // exact threshold key (FP32 key of the K-th entry)
  float pad_f;
  unsigned long long tie_max; // among keys equal to tau, keep packed (i, j) <= tie_max
};

// order-preserving map of FP32 keys to unsigned integers
__device__ __forceinline__ unsigned int key_order(float x) {
  const unsigned int b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}


// One set of launchers per (precision policy, cost kind).
struct PassSet {
  bool mixed;
  // the Sinkhorn half-steps return the number of kernels they launched
  int (*row_lse)(const PassArgs&, const TileGeom&, const MergeWS&, double* F_out,
                 double* out_res, cudaStream_t);
  int (*col_lse)(const PassArgs&, const TileGeom&, const MergeWS&, double* G_out,
                 cudaStream_t);
  void (*marg)(const PassArgs&, const TileGeom&, const MergeWS&, const TrialArgs*,
               double* r, double* c, double* out4, cudaStream_t);
  void (*cert)(const PassArgs&, const TileGeom&, const MergeWS&, const CertArgs&, bool colpass,
               cudaStream_t);
  void (*key_hist)(const PassArgs&, const SparsifyState*, unsigned int* hist, int blocks,
                   cudaStream_t);
  void (*key_compact)(const PassArgs&, SparsifyState*, double* cand_key, long long* cand_idx,
                      int* rowcnt, int blocks, cudaStream_t);
  void (*key_write)(const PassArgs&, const SparsifyState*, const int* indptr, int* indices,
                    double* data, int blocks, cudaStream_t);
  // one-pass candidate collection (mixed policy only; nullptr otherwise)
  void (*fast_collect)(const PassArgs&, float tau_guess, FastSelState*, float* ckey,
                       unsigned long long* cij, int blocks, cudaStream_t);
  // support-tree dual of the certificate from a CSR of the largest entries
  void (*tree_duals)(const PassArgs&, const int* indptr, const int* indices, int ne,
                     const TreeWS&, double* uT, int* err, cudaStream_t);
};

const PassSet* passes_f64(int kind);
const PassSet* passes_mixed(int kind);


// sparse/vector launchers (pins_sparse.cu, pins_select.cu)
struct SparseWS {
  int* rowcnt; int* colcnt;     // m, n
  int* indptr; int* indices; double* data;    // CSR: m+1, cap, cap
  int* colptr; int* rowidx; double* cdata;    // CSC: n+1, cap, cap
  int* trow; double* tval;       // CSC placement before the per-column sort: cap, cap
  int* tcol; double* tcval;      // CSR placement before the per-row sort (one-pass selection)
  int* longseg; int* nlong;      // segments longer than a warp sorts: m + n tags, count
};
void build_csc_from_csr(const int* indptr, const int* indices, const double* data, int m, int n,
                        int nnz, const SparseWS& sw, cudaStream_t st);
void launch_scan(int* cnt, int* ptr, int len, cudaStream_t st);
// CSR + CSC of the entries kept by the one-pass selection (no-op when it failed)
void build_sparse_from_candidates(const FastSelState* fs, const float* ckey,
                                  const unsigned long long* cij, int m, int n, int keep,
                                  const SparseWS& sw, cudaStream_t st);
cudaError_t launch_fast_select(FastSelState* fs, const float* ckey, const unsigned long long* cij,
                               int K, cudaStream_t s);
cudaError_t launch_pcg(int m, int n, double eta, const double* r, const double* c,
                       const int* indptr, const int* indices, const double* data,
                       const int* colptr, const int* rowidx, const double* cdata,
                       const double* rhs, double* x, double* res, double* p, double* q,
                       double* part, double rtol, int max_iter, double* info, int* flag,
                       int sms, cudaStream_t st);
int cg_blocks(int N, int sms);
// single-reduction cluster PCG (pins_cg.cu); *used = false when the system does
// not fit one cluster's shared memory
cudaError_t launch_pcg_cluster(int m, int n, double eta, const double* r, const double* c,
                               const int* indptr, const int* indices, const double* data,
                               const int* colptr, const int* rowidx, const double* cdata,
                               const double* rhs, double* x, double rtol, int max_iter,
                               double* info, int* flag, cudaStream_t st, bool* used);
// Double-float CG of the mixed path (one cluster); *used = false when the
// problem does not fit, and then nothing was launched.  rhs == NULL: the
// right-hand side is (ab - (r; c)); dots != NULL receives <rhs, x>, <ab, x>.
// ent_tgt / ent_val / ent_row hold 2 nnz + PINS_DDCG_ENTRY_PAD slots (each CTA
// pads its entries to a whole number of steps of its 256 threads).
#define PINS_DDCG_ENTRY_PAD (16 * 256)
cudaError_t launch_pcg_dd(int m, int n, double eta, const double* r, const double* c,
                          const int* indptr, const int* indices, const double* data,
                          const int* colptr, const int* rowidx, const double* cdata,
                          const double* rhs, double* x, const double* ab, double* dots,
                          int* ent_tgt, float2* ent_val, int* ent_row, float* ug, int nnz,
                          double rtol, int max_iter, double* info, int* flag, cudaStream_t st,
                          bool* used);
void launch_prep(const double* F, const double* G, int m, int n, double eta, double s,
                 double* A64, double* B64, float2* Add, float2* Bdd, cudaStream_t st);
void launch_trial_prep(const double* d, int m, int n, double scale, double* P64, double* Q64,
                       float2* Pdd, float2* Qdd, cudaStream_t st);
void launch_log_ab(const double* a, const double* b, int m, int n, double* out, cudaStream_t st);
void launch_grad(const double* a, const double* b, const double* r, const double* c, int m,
                 int n, double* g, cudaStream_t st);
void launch_axpy_prep(double* F, double* G, const double* d, int m, int n, double alpha,
                      double eta, double s, double* A64, double* B64, float2* Add, float2* Bdd,
                      cudaStream_t st);
void launch_outer(double* F, double* G, double* Phi, double* Psi, int m, int n, cudaStream_t st);
void launch_dot2(const double* x1, const double* y1, const double* x2, const double* y2, int N,
                 double* out, cudaStream_t st);
void launch_cert_pre(const double* a, const double* r, const double* F, int m, double s,
                     double eta, double* xs, double* u, cudaStream_t st);
void launch_cert_mid(const double* b, const double* c1, int n, double* ys, double* ec,
                     cudaStream_t st);
// out4 = {cost, UB, LB, gap} with LB the larger of the two dual bounds; lb2 (may be
// NULL) = {entropic-dual bound, support-tree bound}
void launch_cert_final(const double* a, const double* b, const double* rr, const double* cr,
                       const double* cp, const double* tc, const double* u2, const double* v,
                       const double* u2T, const double* vT, int m, int n, double* out4,
                       double* lb2, cudaStream_t st);
void launch_d2f(const double* x, float* y, size_t N, cudaStream_t st);
void launch_f2d(const float* x, double* y, size_t N, cudaStream_t st);

// sparsify selection (pins_select.cu)
void launch_key_select(SparsifyState* st, unsigned int* hist, long long total, cudaStream_t s);
cudaError_t launch_cand_select(SparsifyState* st, const double* cand_key,
                               const long long* cand_idx, int n, int* rowcnt, cudaStream_t s);

}  // namespace pins
