// Sinkhorn warm-up half-steps of the mixed policy on a grid cost (Algorithm 2
// warm-up loop), in two separable stages.
//
// Both measures live on one s1 x s2 grid and the raw cost is
// c_ij = (i1 - j1)^2 + (i2 - j2)^2, so a row's base-2 log-sum-exp splits into
// two one-dimensional ones (exact in real arithmetic):
//   LSE2_j (V_j - k c_ij) = LSE2_{j1} ( -k (i1 - j1)^2 + T[j1][i2] ),
//   T[j1][i2]             = LSE2_{j2} ( V_{j1 j2} - k (i2 - j2)^2 ),
// with k = log2(e) kappa (double-float) and V = log2(e) G / eta (row half-step)
// or log2(e) (F / eta - s) (column half-step; c is symmetric).  A half-step
// then costs s1 s2 (s1 + s2) terms instead of (s1 s2)^2.
//
// Stage 1 (k_grid_lse1): CTA q1 holds grid row q1 of V and forms T[q1][p2] for
// every p2 as a base-2 (M, S) pair: M the largest FP32 high part of the
// double-float exponents, S = sum 2^((w_hi - M) + w_lo) in FP32.
// Stage 2 (k_grid_lse2): CTA p2 holds column p2 of T and forms, for every p1,
// sum over q1 of S_q1 2^(M_q1 - k (p1 - q1)^2) as a running (M, S) pair, whose
// M + log2 S is the row's LSE; the potential (and, for the row half-step, the
// l1 row residual of the potentials it replaces) follow as in the streamed
// kernels.  Each term is one FP32 ex2 of a
// double-float exponent, as in the streamed passes; every sum runs in a fixed
// order, so results do not depend on scheduling.
#pragma once

namespace pins {

template <bool ROW>
__device__ __forceinline__ float2 grid_v(const PassArgs& p, int v) {
  if constexpr (ROW) return ddv_mul(split_f64(p.G[v], 0), p.l2e_eta);
  else return a2_of(p, v);
}

// Each output is formed by a group of PINS_GLSE_L lanes (4 outputs per warp):
// lane `sub` of the group takes the terms sub, sub + L, ...; the group's (M, S)
// pairs are then merged in a fixed butterfly over the group.
#define PINS_GLSE_L 8
__device__ __forceinline__ void lse2_group(float& M, float& S) {
#pragma unroll
  for (int o = PINS_GLSE_L / 2; o > 0; o >>= 1) {
    const float Mo = __shfl_xor_sync(0xffffffffu, M, o);
    const float So = __shfl_xor_sync(0xffffffffu, S, o);
    lse2_merge(M, S, Mo, So);
  }
}
// four weighted entries into a running base-2 (M, S): S += sum y_q 2^(w_q)
__device__ __forceinline__ void lse2_chunk_w(float& M, float& S, const float wh[4],
                                             const float wl[4], const float y[4]) {
  const float Mn = fmaxf(M, fmaxf(fmaxf(wh[0], wh[1]), fmaxf(wh[2], wh[3])));
  float t = __fmul_rn(S, ex2_ftz(__fsub_rn(M, Mn)));
#pragma unroll
  for (int q = 0; q < 4; ++q)
    t = __fmaf_rn(y[q], ex2_ftz(__fadd_rn(__fsub_rn(wh[q], Mn), wl[q])), t);
  S = t;
  M = Mn;
}
// log2 of a positive FP32 value in [1, 2^24) as the exponent plus log2 of the
// significand in [1, 2) (absolute error ~1e-7)
__device__ __forceinline__ double log2_split(float S) {
  int e;
  const float f = frexpf(S, &e);          // S = f 2^e, f in [0.5, 1)
  return (double)(e - 1) + (double)log2f(2.f * f);
}

template <bool ROW>
__global__ void __launch_bounds__(PINS_TPB) k_grid_lse1(PassArgs p, int s1, int s2, double* T) {
  extern __shared__ __align__(16) float2 sV[];   // V of grid row q1 (s2 pairs)
  const int q1 = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / PINS_GLSE_L, sub = lane % PINS_GLSE_L;
  constexpr int PER_WARP = 32 / PINS_GLSE_L;
  const float kh = p.kappa2_dd.hi, kl = p.kappa2_dd.lo;
  for (int q2 = threadIdx.x; q2 < s2; q2 += PINS_TPB) sV[q2] = grid_v<ROW>(p, q1 * s2 + q2);
  __syncthreads();
  for (int base = warp * PER_WARP; base < s2; base += PINS_WARPS * PER_WARP) {
    const int p2 = base + grp;
    float M = -INFINITY, S = 0.f;
    if (p2 < s2) {
      int q2 = sub;
      for (; q2 + 3 * PINS_GLSE_L < s2; q2 += 4 * PINS_GLSE_L) {
        float wh[4], wl[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int d = p2 - (q2 + t * PINS_GLSE_L);
          dd_w(sV[q2 + t * PINS_GLSE_L], (float)(d * d), kh, kl, wh[t], wl[t]);
        }
        lse2_chunk(M, S, wh, wl);
      }
      for (; q2 < s2; q2 += PINS_GLSE_L) {
        const int d = p2 - q2;
        float wh, wl;
        dd_w(sV[q2], (float)(d * d), kh, kl, wh, wl);
        lse2_one(M, S, wh, wl);
      }
    }
    lse2_group(M, S);
    if (p2 < s2 && sub == 0) store_f2(T + (size_t)q1 * s2 + p2, M, S);
  }
}

template <bool ROW>
__global__ void __launch_bounds__(PINS_TPB) k_grid_lse2(PassArgs p, int s1, int s2,
                                                        const double* T, MergeWS ws,
                                                        double* out, double* out_res) {
  extern __shared__ __align__(16) float2 sT[];   // (M, S) of T[q1][p2], q1 < s1
  __shared__ double sh_red[PINS_WARPS];
  const int p2 = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / PINS_GLSE_L, sub = lane % PINS_GLSE_L;
  constexpr int PER_WARP = 32 / PINS_GLSE_L;
  const float kh = p.kappa2_dd.hi, kl = p.kappa2_dd.lo;
  const double LN2 = 0.69314718055994530942, L2E = 1.4426950408889634074;
  for (int q1 = threadIdx.x; q1 < s1; q1 += PINS_TPB) sT[q1] = load_f2_cg(T + (size_t)q1 * s2 + p2);
  __syncthreads();
  double res = 0.0;
  for (int base = warp * PER_WARP; base < s1; base += PINS_WARPS * PER_WARP) {
    const int p1 = base + grp;
    float M = -INFINITY, S = 0.f;
    if (p1 < s1) {
      int q1 = sub;
      for (; q1 + 3 * PINS_GLSE_L < s1; q1 += 4 * PINS_GLSE_L) {
        float wh[4], wl[4], y[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int d = p1 - (q1 + t * PINS_GLSE_L);
          const float2 tq = sT[q1 + t * PINS_GLSE_L];
          dd_w(make_float2(tq.x, 0.f), (float)(d * d), kh, kl, wh[t], wl[t]);
          y[t] = tq.y;
        }
        lse2_chunk_w(M, S, wh, wl, y);
      }
      for (; q1 < s1; q1 += PINS_GLSE_L) {
        const int d = p1 - q1;
        const float2 tq = sT[q1];
        float wh, wl;
        dd_w(make_float2(tq.x, 0.f), (float)(d * d), kh, kl, wh, wl);
        const float Mn = fmaxf(M, wh);
        S = __fmaf_rn(tq.y, ex2_ftz(__fadd_rn(__fsub_rn(wh, Mn), wl)),
                      __fmul_rn(S, ex2_ftz(__fsub_rn(M, Mn))));
        M = Mn;
      }
    }
    lse2_group(M, S);
    // the group's first lane writes the potential; only FP64 adds and
    // multiplies here (log a, log b precomputed): a transcendental FP64 call
    // would occupy this GPU's FP64 pipe for thousands of cycles
    if (p1 < s1 && sub == 0) {
      const int i = p1 * s2 + p2;
      const double lse2 = (double)M + log2_split(S);
      if constexpr (ROW) {
        // l1 row residual of the replaced potentials: r_i - a_i = a_i (2^delta - 1)
        // with delta = log2(r_i / a_i)
        if (out_res) {
          const double delta = (p.F[i] * p.inv_eta - p.s) * L2E + lse2 - p.la[i] * L2E;
          const double ai = p.a[i];
          const float dl = (float)(delta * LN2);
          res += (fabs(delta) < 60.0) ? fabs(ai * (double)expm1f(dl)) : fabs(ai * exp2(delta) - ai);
        }
        out[i] = p.eta * (p.la[i] + p.s - LN2 * lse2);
      } else {
        out[i] = p.eta * (p.lb[i] - LN2 * lse2);
      }
    }
  }
  if (ROW && out_res) {   // uniform over the launch
    const double br = block_sum(res, sh_red);
    if (threadIdx.x == 0) ws.scal_row[p2] = br;
    if (arrive_last(ws.cnt_all, (unsigned)s2)) {
      double v = 0.0;
      for (int q = threadIdx.x; q < s2; q += PINS_TPB) v += __ldcg(ws.scal_row + q);
      const double t = block_sum(v, sh_red);
      if (threadIdx.x == 0) *out_res = t;
    }
  }
}

}  // namespace pins
