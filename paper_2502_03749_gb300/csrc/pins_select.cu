// Single-CTA selection kernels of Sparsify (reading R5): threshold-bin search
// over the key histogram, then an exact (key desc, index asc) order of the
// threshold-bin candidates, which fixes the exact threshold (tau, tau_idx).
#include "pins_sparsify.cuh"
#include "pins_kernels.h"

namespace pins {

// 1024 threads: inclusive scan of the 2048 bins (two per thread), then the first
// bin whose cumulative count (plus the entries above the window) reaches K.
__global__ void __launch_bounds__(1024) k_key_select(SparsifyState* st, unsigned int* hist) {
  __shared__ long long sc[1024];
  __shared__ int s_found;
  if (st->done) return;
  const int t = threadIdx.x;
  const unsigned int h0 = hist[2 * t], h1 = hist[2 * t + 1];
  hist[2 * t] = 0u; hist[2 * t + 1] = 0u;          // ready for the next level
  sc[t] = (long long)h0 + h1;
  if (t == 0) s_found = PINS_HIST_NB;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    long long add = (t >= o) ? sc[t - o] : 0;
    __syncthreads();
    sc[t] += add;
    __syncthreads();
  }
  const long long base = st->count_in;
  const long long keep = st->keep;
  const long long excl = base + sc[t] - ((long long)h0 + h1);
  if (excl + h0 >= keep && excl < keep) atomicMin(&s_found, 2 * t);
  else if (excl + h0 + h1 >= keep && excl + h0 < keep) atomicMin(&s_found, 2 * t + 1);
  __syncthreads();
  // the thread owning the found bin updates the state
  const int f = s_found;
  if (f < PINS_HIST_NB && (f >> 1) == t) {
    const long long before = (f & 1) ? excl + h0 : excl;
    const unsigned int cnt = (f & 1) ? h1 : h0;
    if (cnt <= PINS_CAND_CAP || st->level >= 12) {
      st->done = 1;
      st->thr_bin = f;
      st->need = (int)(keep - before);
    } else {   // refine inside the threshold bin
      st->lo = st->lo + (double)f / st->inv_width;
      st->inv_width = st->inv_width * PINS_HIST_NB;
      st->lo_f = (float)st->lo;
      st->inv_width_f = (float)st->inv_width;
      st->count_in = before;
      st->level += 1;
    }
  } else if (f == PINS_HIST_NB && t == 1023) {   // K-th key below the window: widen
    st->count_in = base + sc[1023];
    st->lo = st->lo + (double)PINS_HIST_NB / st->inv_width;
    st->inv_width = st->inv_width / PINS_HIST_NB;
    st->lo_f = (float)st->lo;
    st->inv_width_f = (float)st->inv_width;
    st->level += 1;
    if (st->level >= 12) { st->done = 1; st->overflow = 1; }
  }
}

// one CTA (1024 threads): bitonic sort of the candidates by (key desc, index
// asc); the first `need` are kept: their rows are counted into rowcnt and the
// last one is the exact threshold (tau, tau_idx).
__global__ void __launch_bounds__(1024)
k_cand_select(SparsifyState* st, const double* cand_key, const long long* cand_idx, int n,
              int* rowcnt) {
  extern __shared__ unsigned char smem_raw[];
  double* sk = reinterpret_cast<double*>(smem_raw);
  long long* si = reinterpret_cast<long long*>(sk + PINS_CAND_CAP);
  if (!st->done || st->overflow) return;
  unsigned int cnt = st->cand_count;
  if (cnt > PINS_CAND_CAP) cnt = PINS_CAND_CAP;
  unsigned int P2 = 1;
  while (P2 < cnt) P2 <<= 1;
  for (unsigned int q = threadIdx.x; q < P2; q += blockDim.x) {
    if (q < cnt) { sk[q] = cand_key[q]; si[q] = cand_idx[q]; }
    else { sk[q] = -INFINITY; si[q] = 0x7fffffffffffffffLL; }
  }
  __syncthreads();
  // "a before b" iff key_a > key_b or (key_a == key_b and idx_a < idx_b)
  for (unsigned int k = 2; k <= P2; k <<= 1) {
    for (unsigned int jv = k >> 1; jv > 0; jv >>= 1) {
      for (unsigned int t = threadIdx.x; t < P2; t += blockDim.x) {
        unsigned int l = t ^ jv;
        if (l > t) {
          bool up = ((t & k) == 0);
          double ka = sk[t], kb = sk[l];
          long long ia = si[t], ib = si[l];
          bool a_first = (ka > kb) || (ka == kb && ia < ib);
          if (up ? !a_first : a_first) { sk[t] = kb; sk[l] = ka; si[t] = ib; si[l] = ia; }
        }
      }
      __syncthreads();
    }
  }
  const int need = st->need;
  for (int q = threadIdx.x; q < need && q < (int)cnt; q += blockDim.x)
    atomicAdd(rowcnt + (int)(si[q] / n), 1);
  if (threadIdx.x == 0) {
    if (need >= 1 && need <= (int)cnt) { st->tau = sk[need - 1]; st->tau_idx = si[need - 1]; }
    else st->overflow = 1;
  }
}

void launch_key_select(SparsifyState* st, unsigned int* hist, long long, cudaStream_t s) {
  k_key_select<<<1, 1024, 0, s>>>(st, hist);
}

cudaError_t launch_cand_select(SparsifyState* st, const double* cand_key,
                               const long long* cand_idx, int n, int* rowcnt, cudaStream_t s) {
  size_t smem = (size_t)PINS_CAND_CAP * (sizeof(double) + sizeof(long long));
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_cand_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k_cand_select<<<1, 1024, smem, s>>>(st, cand_key, cand_idx, n, rowcnt);
  return cudaGetLastError();
}

}  // namespace pins
