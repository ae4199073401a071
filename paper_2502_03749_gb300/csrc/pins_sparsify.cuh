// Sparsify kernels of PINS (threshold selection and ordered CSR output).
#pragma once
#include "pins_passes.cuh"
#include "pins_kernels.h"

namespace pins {

// ========================================================================= //
// Sparsify passes (reading R5).  Ranking key: FP64 path k = (F_i + G_j) -
//    s (C_ij + eta) with no contraction; mixed path k = FP32 value of z_ij.
//    Window/binning: u = kref - k; bin = floor((u - lo) * inv_width), bins < 0
//    are above the window (definitely kept), bins >= NB below it.  The bin map
//    is monotone in k, so counts and the final selection agree exactly.
// ========================================================================= //
#define PINS_HIST_NB 2048
#define PINS_CAND_CAP 8192

struct SparsifyState {      // device-resident, written by the select kernels
  double kref, lo, inv_width;   // current window (FP64 keys)
  float kref_f, lo_f, inv_width_f, pad_f;  // the same window for FP32 keys
  long long count_in;       // entries known to be above the window
  int level;
  int done;                 // 1: threshold bin fits the candidate buffer
  int need;                 // entries to take from the threshold bin
  int thr_bin;              // threshold bin
  unsigned int cand_count;  // candidates collected
  int overflow;             // error flag (candidate overflow)
  int keep;                 // K
  int pad_i;
  double tau; long long tau_idx;  // exact threshold (key, linear index)
};

template <class P> struct KeyOf { using T = double; };
template <int K> struct KeyOf<PolMixed<K>> { using T = float; };

template <class P>
__device__ __forceinline__ typename KeyOf<P>::T rank_key(const PassArgs& p, int i, int j) {
  if constexpr (!P::MIXED) {
    double c = P::cost(p, i, j);
    return __dsub_rn(__dadd_rn(p.F[i], p.G[j]), __dmul_rn(p.s, __dadd_rn(c, p.eta)));
  } else {
    float wh, wl, zh, zl;
    dd_w(P::col(p, j), P::cost(p, i, j), p.kappa_dd.hi, p.kappa_dd.lo, wh, wl);
    dd_z(P::row(p, i), wh, wl, zh, zl);
    return __fadd_rn(zh, zl);
  }
}

// keys of entries (i, jb .. jb+3) on the mixed path, A = A_i; -inf past n
template <class P>
__device__ __forceinline__ void keys4_mixed(const PassArgs& p, float2 A, int i, int jb,
                                            float k[4]) {
  float c[4];
  cost4<P>(p, i, jb, p.n, c);
  float2 B[4];
  if (jb + 3 < p.n) {
    const float4 b01 = *reinterpret_cast<const float4*>(p.Bdd + jb);
    const float4 b23 = *reinterpret_cast<const float4*>(p.Bdd + jb + 2);
    B[0] = make_float2(b01.x, b01.y); B[1] = make_float2(b01.z, b01.w);
    B[2] = make_float2(b23.x, b23.y); B[3] = make_float2(b23.z, b23.w);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) B[q] = (jb + q < p.n) ? p.Bdd[jb + q] : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float wh, wl, zh, zl;
    dd_w(B[q], c[q], p.kappa_dd.hi, p.kappa_dd.lo, wh, wl);
    dd_z(A, wh, wl, zh, zl);
    k[q] = (jb + q < p.n) ? __fadd_rn(zh, zl) : -INFINITY;
  }
}

__device__ __forceinline__ int key_bin(double key, const SparsifyState& st) {
  double b = floor(__dmul_rn(__dsub_rn(__dsub_rn(st.kref, key), st.lo), st.inv_width));
  if (b < 0.0) return -1;
  if (b >= (double)PINS_HIST_NB) return PINS_HIST_NB;
  return (int)b;
}
__device__ __forceinline__ int key_bin(float key, const SparsifyState& st) {
  float b = floorf(__fmul_rn(__fsub_rn(__fsub_rn(st.kref_f, key), st.lo_f), st.inv_width_f));
  if (b < 0.0f) return -1;
  if (b >= (float)PINS_HIST_NB) return PINS_HIST_NB;
  return (int)b;
}

// histogram of the keys inside the current window (skipped once done)
template <class P>
__global__ void __launch_bounds__(PINS_TPB)
k_key_hist(PassArgs p, const SparsifyState* __restrict__ st_, unsigned int* hist) {
  __shared__ unsigned int sh[PINS_HIST_NB + 1];
  const SparsifyState st = *st_;
  if (st.done) return;
  for (int q = threadIdx.x; q <= PINS_HIST_NB; q += PINS_TPB) sh[q] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int wpb = PINS_TPB / 32;
  for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < p.m; i += gridDim.x * wpb) {
    if constexpr (P::MIXED) {
      const float2 A = p.Add[i];
#pragma unroll 2
      for (int jb = 4 * lane; jb < p.n; jb += 128) {
        float k[4];
        keys4_mixed<P>(p, A, i, jb, k);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int b = key_bin(k[q], st);
          if (b >= 0 && b < PINS_HIST_NB) atomicAdd(&sh[b], 1u);
        }
      }
    } else {
#pragma unroll 8
      for (int j = lane; j < p.n; j += 32) {
        int b = key_bin(rank_key<P>(p, i, j), st);
        if (b >= 0 && b < PINS_HIST_NB) atomicAdd(&sh[b], 1u);
      }
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < PINS_HIST_NB; q += PINS_TPB)
    if (sh[q]) atomicAdd(&hist[q], sh[q]);
}

// candidates of the threshold bin, and per-row counts of entries above it
template <class P>
__global__ void __launch_bounds__(PINS_TPB)
k_key_compact(PassArgs p, SparsifyState* st_, double* cand_key, long long* cand_idx,
              int* rowcnt) {
  const SparsifyState st = *st_;
  if (!st.done || st.overflow) return;
  const int lane = threadIdx.x & 31;
  const int wpb = PINS_TPB / 32;
  for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < p.m; i += gridDim.x * wpb) {
    int above = 0;
    auto take = [&](auto k, int j) {
      int b = key_bin(k, st);
      above += (b < st.thr_bin) ? 1 : 0;
      if (b == st.thr_bin) {
        unsigned int pos = atomicAdd(&st_->cand_count, 1u);
        if (pos < PINS_CAND_CAP) { cand_key[pos] = (double)k; cand_idx[pos] = (long long)i * p.n + j; }
        else st_->overflow = 1;
      }
    };
    if constexpr (P::MIXED) {
      const float2 A = p.Add[i];
#pragma unroll 2
      for (int jb = 4 * lane; jb < p.n; jb += 128) {
        float k[4];
        keys4_mixed<P>(p, A, i, jb, k);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (jb + q < p.n) take(k[q], jb + q);
      }
    } else {
#pragma unroll 8
      for (int j = lane; j < p.n; j += 32) take(rank_key<P>(p, i, j), j);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) above += __shfl_xor_sync(0xffffffffu, above, o);
    if (lane == 0) rowcnt[i] = above;
  }
}

// CSR of the kept entries, written row by row in column order: an entry is kept
// iff key > tau, or key == tau and its linear index <= tau_idx.
template <class P>
__global__ void __launch_bounds__(PINS_TPB)
k_key_write(PassArgs p, const SparsifyState* __restrict__ st_, const int* __restrict__ indptr,
            int* indices, double* data) {
  const SparsifyState st = *st_;
  const int lane = threadIdx.x & 31;
  const int wpb = PINS_TPB / 32;
  const unsigned int lt = (1u << lane) - 1u;
  // tau in the key's own type (exact: it is one of the keys), so the per-entry
  // test stays off the FP64 pipe on the mixed path
  const typename KeyOf<P>::T tau = (typename KeyOf<P>::T)st.tau;
  for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < p.m; i += gridDim.x * wpb) {
    int pos = indptr[i];
    const int end = indptr[i + 1];
#pragma unroll 4
    for (int j0 = 0; j0 < p.n && pos < end; j0 += 32) {
      const int j = j0 + lane;
      bool keep = false;
      typename KeyOf<P>::T k = 0;
      if (j < p.n) {
        k = rank_key<P>(p, i, j);
        const long long lin = (long long)i * p.n + j;
        keep = (k > tau) || (k == tau && lin <= st.tau_idx);
      }
      unsigned int bal = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        int q = pos + __popc(bal & lt);
        if (q < end) {
          indices[q] = j;
          data[q] = P::MIXED ? exp((double)k) : exp((double)k * p.inv_eta);
        }
      }
      pos += __popc(bal);
    }
  }
}
// candidates of the one-pass selection: keys >= tau_guess, with packed (i, j)
template <class P>
__global__ void __launch_bounds__(PINS_TPB)
k_fast_collect(PassArgs p, float tg, FastSelState* fs, float* ckey, unsigned long long* cij) {
  const int lane = threadIdx.x & 31;
  const int wpb = PINS_TPB / 32;
  const unsigned int lt = (1u << lane) - 1u;
  for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < p.m; i += gridDim.x * wpb) {
    const float2 A = p.Add[i];
#pragma unroll 2
    for (int jb = 4 * lane; jb < p.n; jb += 128) {
      float k[4];
      keys4_mixed<P>(p, A, i, jb, k);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool keep = k[q] >= tg;            // -inf past n never passes
        const unsigned int bal = __ballot_sync(0xffffffffu, keep);
        if (bal) {
          unsigned int base = 0;
          if (lane == 0) base = atomicAdd(&fs->count, (unsigned int)__popc(bal));
          base = __shfl_sync(0xffffffffu, base, 0);
          if (keep) {
            const unsigned int pos = base + __popc(bal & lt);
            if (pos < PINS_FAST_CAP) {
              ckey[pos] = k[q];
              cij[pos] = ((unsigned long long)(unsigned int)i << 32) | (unsigned int)(jb + q);
            }
          }
        }
      }
    }
  }
}

}  // namespace pins
