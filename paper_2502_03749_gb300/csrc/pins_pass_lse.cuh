// Sinkhorn warm-up half-steps (Algorithm 2 warm-up loop; Algorithm 1 in log form).
#pragma once

namespace pins {

// ========================================================================= //
// 1. Row half-step: F_i <- eta (log a_i + s - LSE_j (B_j - kappa C_ij)), and the
//    row residual sum_i |X~(F_old) 1 - a|_i before the update (out_res, may be 0).
// ========================================================================= //
template <class P>
__global__ void __launch_bounds__(PINS_TPB)
k_row_lse(PassArgs p, TileGeom g, MergeWS ws, double* F_out, double* out_res) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = p.m, n = p.n;
  __shared__ double sh_red[PINS_WARPS];
  __shared__ double stg[2][PINS_STAGE];
  const float kh = p.kappa_dd.hi, kl = p.kappa_dd.lo;
  for (int ct = blockIdx.x; ct < g.nct; ct += g.gx) {
    const bool first = (ct == (int)blockIdx.x);
    typename P::Col cd[PINS_CPL];
    int jj[PINS_CPL];
#pragma unroll
    for (int q = 0; q < PINS_CPL; ++q) {
      jj[q] = ct * PINS_TC + lane + 32 * q;
      cd[q] = P::col(p, jj[q] < n ? jj[q] : n - 1);
    }
    for (int rt = blockIdx.y; rt < g.nrt; rt += g.gy) {
#pragma unroll 2
      for (int t = 0; t < PINS_RPT; ++t) {
        const int i = rt * PINS_TR + warp + PINS_WARPS * t;
        if (i >= m) break;
        const size_t k = (size_t)blockIdx.x * m + i;
        if constexpr (!P::MIXED) {
          double v[PINS_CPL];
          double mx = -INFINITY;
#pragma unroll
          for (int q = 0; q < PINS_CPL; ++q) {
            v[q] = (jj[q] < n) ? fma(-p.kappa, P::cost(p, i, jj[q]), cd[q]) : -INFINITY;
            mx = fmax(mx, v[q]);
          }
          mx = warp_maxd(mx);
          double sum = 0.0;
#pragma unroll
          for (int q = 0; q < PINS_CPL; ++q) sum += (jj[q] < n) ? exp(v[q] - mx) : 0.0;
          sum = warp_sum(sum);
          if (lane == 0) {
            if (first) { ws.rowpart0[k] = mx; ws.rowpart1[k] = sum; }
            else {
              double m1 = ws.rowpart0[k], s1 = ws.rowpart1[k];
              lse_merge(m1, s1, mx, sum);
              ws.rowpart0[k] = m1; ws.rowpart1[k] = s1;
            }
          }
        } else {
          float wh[PINS_CPL], wl[PINS_CPL];
          float mx = -INFINITY;
#pragma unroll
          for (int q = 0; q < PINS_CPL; ++q) {
            if (jj[q] < n) dd_w(cd[q], P::cost(p, i, jj[q]), kh, kl, wh[q], wl[q]);
            else { wh[q] = -INFINITY; wl[q] = 0.f; }
            mx = fmaxf(mx, wh[q]);
          }
          mx = warp_maxf(mx);
          float sum = 0.f;
#pragma unroll
          for (int q = 0; q < PINS_CPL; ++q)
            if (jj[q] < n) sum += exp2f(((wh[q] - mx) + wl[q]) * 1.4426950408889634f);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
          if (lane == 0) {   // (max, sum) kept as a raw float pair
            if (first) store_f2(ws.rowpart0 + k, mx, sum);
            else {
              float2 o = load_f2(ws.rowpart0 + k);
              lse_merge_f(o.x, o.y, mx, sum);
              store_f2(ws.rowpart0 + k, o.x, o.y);
            }
          }
        }
      }
    }
  }
  // merge row partials across strips (last CTA of this row block)
  if (arrive_last(ws.cnt_row + blockIdx.y, g.gx)) {
    double res = 0.0;
    for (int rt = blockIdx.y; rt < g.nrt; rt += g.gy) {
      const int i0 = rt * PINS_TR;
      const int nr = min(PINS_TR, m - i0);
      stage8(ws.rowpart0 + i0, m, g.gx, PINS_TR, nr, stg[0]);
      if (!P::MIXED) stage8(ws.rowpart1 + i0, m, g.gx, PINS_TR, nr, stg[1]);
      __syncthreads();
      if ((int)threadIdx.x < nr) {
        const int i = i0 + threadIdx.x;
        double M = -INFINITY, S = 0.0;
        if constexpr (P::MIXED) {
          float Mf = -INFINITY, Sf = 0.f;
          for (int x = 0; x < g.gx; ++x) {
            float2 o = as_f2(stg[0][x * PINS_TR + threadIdx.x]);
            lse_merge_f(Mf, Sf, o.x, o.y);
          }
          M = (double)Mf; S = (double)Sf;
        } else {
          for (int x = 0; x < g.gx; ++x)
            lse_merge(M, S, stg[0][x * PINS_TR + threadIdx.x], stg[1][x * PINS_TR + threadIdx.x]);
        }
        const double lse = M + log(S);
        const double A = P::MIXED ? (double)p.Add[i].x + (double)p.Add[i].y : p.A64[i];
        const double ai = p.a[i];
        if (out_res) res += fabs(exp(A + lse) - ai);
        F_out[i] = p.eta * (log(ai) + p.s - lse);
      }
      __syncthreads();
    }
    const double br = block_sum(res, sh_red);
    if (threadIdx.x == 0) ws.scal_row[blockIdx.y] = br;
  }
  if (out_res && arrive_last(ws.cnt_all, g.gx * g.gy)) {   // residual only when asked for
    const double v = ((int)threadIdx.x < g.gy) ? __ldcg(ws.scal_row + threadIdx.x) : 0.0;
    const double t = block_sum(v, sh_red);
    if (threadIdx.x == 0 && out_res) *out_res = t;
  }
}

// ========================================================================= //
// 2. Column half-step (new F): G_j <- eta (log b_j - LSE_i (A_i - kappa C_ij)).
// ========================================================================= //
template <class P>
__global__ void __launch_bounds__(PINS_TPB)
k_col_lse(PassArgs p, TileGeom g, MergeWS ws, double* G_out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = p.m, n = p.n;
  __shared__ double stg[2][PINS_STAGE];
  const float kh = p.kappa_dd.hi, kl = p.kappa_dd.lo;
  for (int ct = blockIdx.x; ct < g.nct; ct += g.gx) {
    int jj[PINS_CPL];
#pragma unroll
    for (int q = 0; q < PINS_CPL; ++q) jj[q] = ct * PINS_TC + lane + 32 * q;
    double cM[PINS_CPL], cS[PINS_CPL];   // FP64 policy running (max, sum)
    float fM[PINS_CPL], fS[PINS_CPL];    // mixed policy running (max, sum), FP32 only
#pragma unroll
    for (int q = 0; q < PINS_CPL; ++q) { cM[q] = -INFINITY; cS[q] = 0.0; fM[q] = -INFINITY; fS[q] = 0.f; }
    for (int rt = blockIdx.y; rt < g.nrt; rt += g.gy) {
      if constexpr (!P::MIXED) {
        double v[PINS_RPT][PINS_CPL];
        double mx[PINS_CPL];
#pragma unroll
        for (int q = 0; q < PINS_CPL; ++q) mx[q] = -INFINITY;
#pragma unroll
        for (int t = 0; t < PINS_RPT; ++t) {
          const int i = rt * PINS_TR + warp + PINS_WARPS * t;
          const double A = (i < m) ? P::row(p, i) : 0.0;
#pragma unroll
          for (int q = 0; q < PINS_CPL; ++q) {
            v[t][q] = (i < m && jj[q] < n) ? fma(-p.kappa, P::cost(p, i, jj[q]), A) : -INFINITY;
            mx[q] = fmax(mx[q], v[t][q]);
          }
        }
#pragma unroll
        for (int q = 0; q < PINS_CPL; ++q) {
          if (mx[q] == -INFINITY) continue;
          double s = 0.0;
#pragma unroll
          for (int t = 0; t < PINS_RPT; ++t) s += exp(v[t][q] - mx[q]);
          lse_merge(cM[q], cS[q], mx[q], s);
        }
      } else {
        float wh[PINS_RPT][PINS_CPL], wl[PINS_RPT][PINS_CPL];
        float mx[PINS_CPL];
#pragma unroll
        for (int q = 0; q < PINS_CPL; ++q) mx[q] = -INFINITY;
#pragma unroll
        for (int t = 0; t < PINS_RPT; ++t) {
          const int i = rt * PINS_TR + warp + PINS_WARPS * t;
          const float2 A = (i < m) ? P::row(p, i) : make_float2(0.f, 0.f);
#pragma unroll
          for (int q = 0; q < PINS_CPL; ++q) {
            if (i < m && jj[q] < n) dd_w(A, P::cost(p, i, jj[q]), kh, kl, wh[t][q], wl[t][q]);
            else { wh[t][q] = -INFINITY; wl[t][q] = 0.f; }
            mx[q] = fmaxf(mx[q], wh[t][q]);
          }
        }
#pragma unroll
        for (int q = 0; q < PINS_CPL; ++q) {
          if (mx[q] == -INFINITY) continue;
          float s = 0.f;
#pragma unroll
          for (int t = 0; t < PINS_RPT; ++t)
            if (wh[t][q] != -INFINITY) s += exp2f(((wh[t][q] - mx[q]) + wl[t][q]) * 1.4426950408889634f);
          lse_merge_f(fM[q], fS[q], mx[q], s);
        }
      }
    }
    // combine the 8 warps of this CTA per column (stg reused as [warp][column])
    __syncthreads();
    if constexpr (P::MIXED) {
#pragma unroll
      for (int q = 0; q < PINS_CPL; ++q) {
        float2 v = make_float2(fM[q], fS[q]);
        stg[0][warp * PINS_TC + lane + 32 * q] = *reinterpret_cast<double*>(&v);
      }
      __syncthreads();
      for (int c = threadIdx.x; c < PINS_TC; c += PINS_TPB) {
        float M = -INFINITY, S = 0.f;
        for (int w = 0; w < PINS_WARPS; ++w) {
          float2 o = as_f2(stg[0][w * PINS_TC + c]);
          lse_merge_f(M, S, o.x, o.y);
        }
        const int j = ct * PINS_TC + c;
        if (j < n) store_f2(ws.colpart0 + (size_t)blockIdx.y * n + j, M, S);
      }
    } else {
#pragma unroll
      for (int q = 0; q < PINS_CPL; ++q) {
        stg[0][warp * PINS_TC + lane + 32 * q] = cM[q];
        stg[1][warp * PINS_TC + lane + 32 * q] = cS[q];
      }
      __syncthreads();
      for (int c = threadIdx.x; c < PINS_TC; c += PINS_TPB) {
        double M = -INFINITY, S = 0.0;
        for (int w = 0; w < PINS_WARPS; ++w) lse_merge(M, S, stg[0][w * PINS_TC + c], stg[1][w * PINS_TC + c]);
        const int j = ct * PINS_TC + c;
        if (j < n) {
          ws.colpart0[(size_t)blockIdx.y * n + j] = M;
          ws.colpart1[(size_t)blockIdx.y * n + j] = S;
        }
      }
    }
    __syncthreads();
  }
  // merge column partials across row blocks (last CTA of this strip), staged
  // 16 row blocks at a time
  if (arrive_last(ws.cnt_col + blockIdx.x, g.gy)) {
    for (int ct = blockIdx.x; ct < g.nct; ct += g.gx) {
      const int j0 = ct * PINS_TC;
      const int nc = min(PINS_TC, n - j0);
      double M = -INFINITY, S = 0.0;
      float Mf = -INFINITY, Sf = 0.f;
      for (int y0 = 0; y0 < g.gy; y0 += 16) {
        const int cnt = min(16, g.gy - y0);
        stage8(ws.colpart0 + (size_t)y0 * n + j0, n, cnt, PINS_TC, nc, stg[0]);
        if (!P::MIXED) stage8(ws.colpart1 + (size_t)y0 * n + j0, n, cnt, PINS_TC, nc, stg[1]);
        __syncthreads();
        if ((int)threadIdx.x < nc) {
          for (int s = 0; s < cnt; ++s) {
            if constexpr (P::MIXED) {
              float2 o = as_f2(stg[0][s * PINS_TC + threadIdx.x]);
              lse_merge_f(Mf, Sf, o.x, o.y);
            } else {
              lse_merge(M, S, stg[0][s * PINS_TC + threadIdx.x], stg[1][s * PINS_TC + threadIdx.x]);
            }
          }
        }
        __syncthreads();
      }
      if ((int)threadIdx.x < nc) {
        if constexpr (P::MIXED) { M = (double)Mf; S = (double)Sf; }
        const int j = j0 + threadIdx.x;
        G_out[j] = p.eta * (log(p.b[j]) - (M + log(S)));
      }
    }
  }
}

}  // namespace pins
