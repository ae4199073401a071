// Sinkhorn warm-up half-steps of the mixed policy (Algorithm 2 warm-up loop;
// Algorithm 1 in log form), streamed with an online log-sum-exp.
//
// Each thread keeps a running (M, S) with S = sum exp(w - M): an entry w below
// M adds exp(w - M); an entry above M first rescales S by exp(M - w) (rare once
// the running maximum has settled).  No tile of w is held in registers and no
// per-tile maximum pass is needed, so the kernels stream C at one FP32 ex2 per
// entry.  w = V - kappa C_ij is formed in double-float and the exponent
// (w_hi - M) + w_lo in FP32, as in the tiled kernels.
//
// Row half-step: CTA (x, y) stages the B_j of column segment x in shared memory;
// warp w takes rows y*8 + w + t*8*gridDim.y over that segment; a warp's (M, S)
// partial per row goes to rowpart0[x*m + i]; the last of the gridDim.x CTAs of
// row group y merges the segments of its rows in segment order.
// Column half-step: CTA (x, y) takes column strips x, x + gridDim.x, ... of 128
// columns and rows [y*rb, (y+1)*rb); lane l owns 4 consecutive columns; the 8
// warps' partials are merged in warp order, then the last of the gridDim.y CTAs
// of a strip merges the row blocks in block order.  Results do not depend on
// scheduling.
#pragma once

namespace pins {

#define PINS_LSE_LOG2E 1.4426950408889634f

__device__ __forceinline__ void lse_online(float& M, float& S, float wh, float wl) {
  float d = __fsub_rn(wh, M);
  if (d > 0.f) {                 // new running maximum (also the first entry: M = -inf)
    S = __fmul_rn(S, exp2f(-d * PINS_LSE_LOG2E));
    M = wh;
    d = 0.f;
  }
  S = __fadd_rn(S, exp2f(__fadd_rn(d, wl) * PINS_LSE_LOG2E));
}

// 4 consecutive raw costs of row i from column j (entries at or beyond jend are
// left unspecified); a 16-byte load when the dense row allows it
template <class P>
__device__ __forceinline__ void cost4(const PassArgs& p, int i, int j, int jend, float c[4]) {
  if constexpr (std::is_same<P, PolMixed<COST_DENSE>>::value) {
    const float* row = p.cost.C32 + (size_t)i * p.n;
    if ((p.n & 3) == 0 && j + 3 < jend) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(row + j));
      c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
      return;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) c[q] = (j + q < jend) ? __ldg(row + j + q) : 0.f;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) c[q] = (j + q < jend) ? P::cost(p, i, j + q) : 0.f;
  }
}

template <class P>
__global__ void __launch_bounds__(PINS_TPB)
k_row_lse_mx(PassArgs p, int seg, MergeWS ws, double* F_out, double* out_res) {
  extern __shared__ float2 sB[];
  __shared__ double sh_red[PINS_WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = p.m, n = p.n;
  const int x = blockIdx.x, y = blockIdx.y, SX = gridDim.x, GY = gridDim.y;
  const int j0 = x * seg, j1 = min(n, j0 + seg);
  const float kh = p.kappa_dd.hi, kl = p.kappa_dd.lo;
  for (int j = j0 + threadIdx.x; j < j1; j += PINS_TPB) sB[j - j0] = p.Bdd[j];
  __syncthreads();
  for (int i = y * PINS_WARPS + warp; i < m; i += GY * PINS_WARPS) {
    float M = -INFINITY, S = 0.f;
    for (int jb = j0 + 4 * lane; jb < j1; jb += 128) {
      float c[4];
      cost4<P>(p, i, jb, j1, c);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (jb + q < j1) {
          float wh, wl;
          dd_w(sB[jb + q - j0], c[q], kh, kl, wh, wl);
          lse_online(M, S, wh, wl);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float Mo = __shfl_xor_sync(0xffffffffu, M, o);
      const float So = __shfl_xor_sync(0xffffffffu, S, o);
      lse_merge_f(M, S, Mo, So);
    }
    if (lane == 0) store_f2(ws.rowpart0 + (size_t)x * m + i, M, S);
  }
  // merge the segments of this row group (last of its SX CTAs)
  if (arrive_last(ws.cnt_row + y, SX)) {
    double res = 0.0;
    const int per = PINS_WARPS * ((m + GY * PINS_WARPS - 1) / (GY * PINS_WARPS));
    for (int k = threadIdx.x; k < per; k += PINS_TPB) {
      const int i = y * PINS_WARPS + (k % PINS_WARPS) + (k / PINS_WARPS) * GY * PINS_WARPS;
      if (i >= m) continue;
      float Mf = -INFINITY, Sf = 0.f;
      for (int xs = 0; xs < SX; ++xs) {
        const float2 o = load_f2_cg(ws.rowpart0 + (size_t)xs * m + i);
        lse_merge_f(Mf, Sf, o.x, o.y);
      }
      const double lse = (double)Mf + log((double)Sf);
      const double A = (double)p.Add[i].x + (double)p.Add[i].y;
      const double ai = p.a[i];
      res += fabs(exp(A + lse) - ai);
      F_out[i] = p.eta * (log(ai) + p.s - lse);
    }
    const double br = block_sum(res, sh_red);
    if (threadIdx.x == 0) ws.scal_row[y] = br;
  }
  if (arrive_last(ws.cnt_all, SX * GY)) {
    double v = 0.0;
    for (int q = threadIdx.x; q < GY; q += PINS_TPB) v += __ldcg(ws.scal_row + q);
    const double t = block_sum(v, sh_red);
    if (threadIdx.x == 0 && out_res) *out_res = t;
  }
}

template <class P>
__global__ void __launch_bounds__(PINS_TPB)
k_col_lse_mx(PassArgs p, int rb, MergeWS ws, double* G_out) {
  __shared__ float2 stg[PINS_WARPS][PINS_TC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = p.m, n = p.n;
  const int i0 = blockIdx.y * rb, i1 = min(m, i0 + rb);
  const int nct = (n + PINS_TC - 1) / PINS_TC;
  const float kh = p.kappa_dd.hi, kl = p.kappa_dd.lo;
  for (int ct = blockIdx.x; ct < nct; ct += gridDim.x) {
    const int jb = ct * PINS_TC + 4 * lane;
    float M[4], S[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) { M[q] = -INFINITY; S[q] = 0.f; }
    int i = i0 + warp;
    // four rows per step: loads first, then the updates
    for (; i + 3 * PINS_WARPS < i1; i += 4 * PINS_WARPS) {
      float c[4][4];
      float2 A[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        A[t] = p.Add[i + t * PINS_WARPS];
        cost4<P>(p, i + t * PINS_WARPS, jb, n, c[t]);
      }
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (jb + q < n) {
            float wh, wl;
            dd_w(A[t], c[t][q], kh, kl, wh, wl);
            lse_online(M[q], S[q], wh, wl);
          }
    }
    for (; i < i1; i += PINS_WARPS) {
      float c[4];
      const float2 A = p.Add[i];
      cost4<P>(p, i, jb, n, c);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (jb + q < n) {
          float wh, wl;
          dd_w(A, c[q], kh, kl, wh, wl);
          lse_online(M[q], S[q], wh, wl);
        }
    }
    // merge the 8 warps per column, in warp order
#pragma unroll
    for (int q = 0; q < 4; ++q) stg[warp][4 * lane + q] = make_float2(M[q], S[q]);
    __syncthreads();
    if (threadIdx.x < PINS_TC) {
      float Mc = -INFINITY, Sc = 0.f;
#pragma unroll
      for (int w = 0; w < PINS_WARPS; ++w) lse_merge_f(Mc, Sc, stg[w][threadIdx.x].x, stg[w][threadIdx.x].y);
      const int j = ct * PINS_TC + threadIdx.x;
      if (j < n) store_f2(ws.colpart0 + (size_t)blockIdx.y * n + j, Mc, Sc);
    }
    __syncthreads();
  }
  // merge the row blocks of this CTA's strips (last of the gridDim.y CTAs)
  if (arrive_last(ws.cnt_col + blockIdx.x, gridDim.y)) {
    for (int ct = blockIdx.x; ct < nct; ct += gridDim.x) {
      const int j = ct * PINS_TC + threadIdx.x;
      if (threadIdx.x < PINS_TC && j < n) {
        float Mf = -INFINITY, Sf = 0.f;
        for (int yb = 0; yb < (int)gridDim.y; ++yb) {
          const float2 o = load_f2_cg(ws.colpart0 + (size_t)yb * n + j);
          lse_merge_f(Mf, Sf, o.x, o.y);
        }
        G_out[j] = p.eta * (log(p.b[j]) - ((double)Mf + log((double)Sf)));
      }
    }
  }
}

}  // namespace pins
