// Single-CTA selection kernels of Sparsify (reading R5): threshold-bin search
// over the key histogram, then an exact (key desc, index asc) order of the
// threshold-bin candidates.
#include "pins_passes.cuh"
#include "pins_kernels.h"

namespace pins {

// one CTA: scan the histogram, find the bin holding the K-th key
__global__ void k_key_select(SparsifyState* st, unsigned int* hist, long long total_entries) {
  __shared__ unsigned int sh[PINS_HIST_NB];
  __shared__ long long s_excl[PINS_HIST_NB];
  if (st->done) return;
  for (int q = threadIdx.x; q < PINS_HIST_NB; q += blockDim.x) { sh[q] = hist[q]; hist[q] = 0u; }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long acc = st->count_in;
    int found = -1;
    for (int q = 0; q < PINS_HIST_NB; ++q) {
      s_excl[q] = acc;
      if (found < 0 && acc + (long long)sh[q] >= st->keep) found = q;
      acc += sh[q];
    }
    if (found >= 0) {
      long long before = s_excl[found];
      unsigned int cnt = sh[found];
      if (cnt <= PINS_CAND_CAP || st->level >= 12) {
        st->done = 1;
        st->thr_bin = found;
        st->need = (int)(st->keep - before);
      } else {   // refine inside the threshold bin
        st->lo = st->lo + found * st->width;
        st->width = st->width / PINS_HIST_NB;
        st->count_in = before;
        st->level += 1;
      }
    } else {     // K-th key lies below the window: widen downwards
      st->count_in = acc;
      st->lo = st->lo + PINS_HIST_NB * st->width;
      st->width = st->width * PINS_HIST_NB;
      st->level += 1;
      if (st->level >= 12) { st->done = 1; st->overflow = 1; }
    }
  }
}

// one CTA (1024 threads): bitonic sort of the candidates by (key desc, index
// asc), append the first `need` to the COO list, record the exact threshold.
__global__ void __launch_bounds__(1024)
k_cand_select(SparsifyState* st, const double* cand_key, const long long* cand_idx,
              double* coo_key, long long* coo_idx, int coo_cap) {
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
  int need = st->need;
  unsigned int base = st->coo_count;
  for (int q = threadIdx.x; q < need; q += blockDim.x) {
    if ((int)(base + q) < coo_cap) { coo_key[base + q] = sk[q]; coo_idx[base + q] = si[q]; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (need > 0) { st->tau = sk[need - 1]; st->tau_idx = si[need - 1]; }
    st->coo_count = base + need;
    if ((int)(base + need) > coo_cap) st->overflow = 1;
  }
}

void launch_key_select(SparsifyState* st, unsigned int* hist, long long total, cudaStream_t s) {
  k_key_select<<<1, 1024, 0, s>>>(st, hist, total);
}

cudaError_t launch_cand_select(SparsifyState* st, const double* cand_key,
                               const long long* cand_idx, double* coo_key, long long* coo_idx,
                               int coo_cap, cudaStream_t s) {
  size_t smem = (size_t)PINS_CAND_CAP * (sizeof(double) + sizeof(long long));
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_cand_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k_cand_select<<<1, 1024, smem, s>>>(st, cand_key, cand_idx, coo_key, coo_idx, coo_cap);
  return cudaGetLastError();
}

}  // namespace pins
