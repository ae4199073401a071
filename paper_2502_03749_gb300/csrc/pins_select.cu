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
  static const cudaError_t configured =   // once, thread-safely
      cudaFuncSetAttribute(k_cand_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (configured != cudaSuccess) return configured;
  k_cand_select<<<1, 1024, smem, s>>>(st, cand_key, cand_idx, n, rowcnt);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------- //
// Exact top-K of the one-pass candidates (one CTA, 1024 threads).  Keys are
// mapped to order-preserving unsigned integers and the K-th largest is found by
// a three-pass radix select (11, 11, 10 bits) over the keys staged in shared
// memory; the entries tied at that key are then ordered by packed (i, j) and the
// first `need` kept, exactly as the histogram path ranks (key desc, index asc).
// Resets fs->count for the next collect pass.
// ------------------------------------------------------------------------- //
__global__ void __launch_bounds__(1024)
k_fast_select(FastSelState* fs, const float* ckey, const unsigned long long* cij, int K) {
  extern __shared__ unsigned int fsm[];
  unsigned int* su = fsm;                                  // PINS_FAST_CAP keys
  unsigned int* hist = su + PINS_FAST_CAP;                 // 2048 bins
  unsigned long long* tie = reinterpret_cast<unsigned long long*>(hist + 2048);  // PINS_FAST_TIES
  __shared__ unsigned int s_digit, s_want, s_nt;
  const int t = threadIdx.x;
  const unsigned int cnt = fs->count;
  __syncthreads();
  if (t == 0) fs->count = 0u;
  if (cnt < (unsigned int)K || cnt > PINS_FAST_CAP) {
    if (t == 0) { fs->fail = (cnt < (unsigned int)K) ? 1 : 2; fs->ncand = 0u; }
    return;
  }
  for (unsigned int q = t; q < cnt; q += 1024) su[q] = key_order(ckey[q]);
  unsigned int prefix = 0u, pmask = 0u, want = (unsigned int)K;
  const int shifts[3] = {21, 10, 0};
  const int widths[3] = {11, 11, 10};
  for (int ps = 0; ps < 3; ++ps) {
    const int sh = shifts[ps];
    const unsigned int nb = 1u << widths[ps];
    for (unsigned int b = t; b < 2048u; b += 1024) hist[b] = 0u;
    if (t == 0) s_digit = 0xffffffffu;
    __syncthreads();
    for (unsigned int q = t; q < cnt; q += 1024) {
      const unsigned int u = su[q];
      if ((u & pmask) == prefix) atomicAdd(&hist[(u >> sh) & (nb - 1u)], 1u);
    }
    __syncthreads();
    if (t < 32) {
      // digits from the top: the first (highest) digit whose cumulative count reaches want
      const unsigned int per = nb / 32u;                   // bins per lane, lane 0 = top bins
      unsigned int loc = 0u;
      for (unsigned int b = 0; b < per; ++b) loc += hist[nb - 1u - (t * per + b)];
      unsigned int inc = loc;                              // inclusive scan over lanes
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (t >= o) inc += v;
      }
      const unsigned int excl = inc - loc;
      const unsigned int hitmask = __ballot_sync(0xffffffffu, excl < want && inc >= want);
      const int owner = __ffs(hitmask) - 1;
      if (t == owner) {
        unsigned int run = excl;
        for (unsigned int b = 0; b < per; ++b) {
          const unsigned int bin = nb - 1u - (t * per + b);
          const unsigned int h = hist[bin];
          if (run + h >= want) { s_digit = bin; s_want = want - run; break; }
          run += h;
        }
      }
    }
    __syncthreads();
    if (s_digit == 0xffffffffu) {                          // counts inconsistent with K
      if (t == 0) { fs->fail = 4; fs->ncand = 0u; }
      return;
    }
    prefix |= s_digit << sh;
    pmask |= (nb - 1u) << sh;
    want = s_want;
    __syncthreads();
  }
  // prefix is the threshold key; `want` entries are needed among the ties
  if (t == 0) s_nt = 0u;
  __syncthreads();
  for (unsigned int q = t; q < cnt; q += 1024) {
    if (su[q] == prefix) {
      const unsigned int pos = atomicAdd(&s_nt, 1u);
      if (pos < PINS_FAST_TIES) tie[pos] = cij[q];
    }
  }
  __syncthreads();
  const unsigned int nt = s_nt;
  if (nt > PINS_FAST_TIES || nt < want) {
    if (t == 0) { fs->fail = 3; fs->ncand = 0u; }
    return;
  }
  unsigned int P2 = 1u;
  while (P2 < nt) P2 <<= 1;
  for (unsigned int q = nt + t; q < P2; q += 1024) tie[q] = ~0ull;
  __syncthreads();
  for (unsigned int k = 2; k <= P2; k <<= 1) {
    for (unsigned int jv = k >> 1; jv > 0; jv >>= 1) {
      for (unsigned int q = t; q < P2; q += 1024) {
        const unsigned int l = q ^ jv;
        if (l > q) {
          const bool up = (q & k) == 0;
          const unsigned long long a = tie[q], b = tie[l];
          if (up ? (a > b) : (a < b)) { tie[q] = b; tie[l] = a; }
        }
      }
      __syncthreads();
    }
  }
  if (t == 0) {
    const unsigned int u = prefix;
    const unsigned int bits = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    fs->tau = __uint_as_float(bits);
    fs->tie_max = tie[want - 1u];
    fs->ncand = cnt;
    fs->fail = 0;
  }
}

cudaError_t launch_fast_select(FastSelState* fs, const float* ckey, const unsigned long long* cij,
                               int K, cudaStream_t s) {
  const size_t smem = sizeof(unsigned int) * (PINS_FAST_CAP + 2048) +
                      sizeof(unsigned long long) * PINS_FAST_TIES;
  static const cudaError_t configured =   // once, thread-safely
      cudaFuncSetAttribute(k_fast_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (configured != cudaSuccess) return configured;
  k_fast_select<<<1, 1024, smem, s>>>(fs, ckey, cij, K);
  return cudaGetLastError();
}

}  // namespace pins
