// m x n pass kernels of PINS, templated on the arithmetic policy (FP64 or
// mixed) and the cost source.  Every pass tiles the matrix into 64 x 128 tiles;
// a CTA owns one column strip x and one row block y and loops over the tiles
// congruent to (x, y).  Row results are merged across strips and column results
// across row blocks by the last CTA to arrive (fixed merge order, so every result
// is bit-reproducible regardless of scheduling or of other work on the device).
#pragma once
#include "pins_common.cuh"

namespace pins {

// ------------------------------------------------------------------------- //
// Policies: how z_ij and its pieces are formed
// ------------------------------------------------------------------------- //
template <int KIND> struct PolF64 {
  static constexpr bool MIXED = false;
  using Row = double;   // A_i = F_i / eta - s
  using Col = double;   // B_j = G_j / eta
  __device__ __forceinline__ static Row row(const PassArgs& p, int i) { return __ldg(p.A64 + i); }
  __device__ __forceinline__ static Col col(const PassArgs& p, int j) { return __ldg(p.B64 + j); }
  // kappa C_ij
  __device__ __forceinline__ static double cost(const PassArgs& p, int i, int j) {
    return Cost64<KIND>::c(p.cost, i, j);
  }
};

template <int KIND> struct PolMixed {
  static constexpr bool MIXED = true;
  using Row = float2;
  using Col = float2;
  __device__ __forceinline__ static Row row(const PassArgs& p, int i) { return p.Add[i]; }
  __device__ __forceinline__ static Col col(const PassArgs& p, int j) { return p.Bdd[j]; }
  __device__ __forceinline__ static float cost(const PassArgs& p, int i, int j) {
    return Cost32<KIND>::c(p.cost, i, j);
  }
};

// w = V - kappa c in double-float (V one of A_i, B_j); returns (hi, lo)
__device__ __forceinline__ void dd_w(float2 V, float c, float kh, float kl, float& wh, float& wl) {
  float ph, pe; two_prod(kh, c, ph, pe);
  pe = __fmaf_rn(kl, c, pe);
  float se; two_sum(V.x, -ph, wh, se);
  wl = __fadd_rn(se, __fsub_rn(V.y, pe));
}
// z = A + w in double-float
__device__ __forceinline__ void dd_z(float2 A, float wh, float wl, float& zh, float& zl) {
  float ze; two_sum(A.x, wh, zh, ze);
  zl = __fadd_rn(ze, __fadd_rn(A.y, wl));
}

// ------------------------------------------------------------------------- //
// arrival helper: returns true in the CTA that arrived last (block-uniform)
// ------------------------------------------------------------------------- //
__device__ __forceinline__ bool arrive_last(unsigned int* counter, unsigned int total) {
  __shared__ unsigned int s_flag;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = atomicAdd(counter, 1u);
    s_flag = (t == total - 1) ? 1u : 0u;
  }
  __syncthreads();
  bool last = s_flag != 0u;
  if (last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;  // ready for the next launch
  }
  return last;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (l < PINS_WARPS) ? sh[l] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;  // valid in thread 0 (and warp 0)
}
__device__ __forceinline__ double block_max(double v, double* sh) {
  v = warp_maxd(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = -INFINITY;
  if (threadIdx.x < 32) {
    r = (l < PINS_WARPS) ? sh[l] : -INFINITY;
    r = warp_maxd(r);
  }
  __syncthreads();
  return r;
}

// ========================================================================= //
// 1. Sinkhorn row half-step (Alg. 2 warm-up, first update):
//    F_i <- eta (log a_i + s - LSE_j (B_j - kappa C_ij)),
//    and the row residual sum_i |X~(F_old) 1 - a|_i before the update.
//    out_res: device double (may be null).
// ========================================================================= //
template <class P>
__global__ void __launch_bounds__(PINS_TPB)
k_row_lse(PassArgs p, TileGeom g, MergeWS ws, double* F_out, double* out_res) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = p.m, n = p.n;
  __shared__ double sh_red[PINS_WARPS];
  float kh = p.kappa_dd.hi, kl = p.kappa_dd.lo;
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
        double M, S;
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
          M = mx; S = sum;
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
          M = (double)mx; S = (double)sum;
        }
        if (lane == 0) {
          size_t k = (size_t)blockIdx.x * m + i;
          if (first) { ws.rowpart0[k] = M; ws.rowpart1[k] = S; }
          else {
            double m1 = ws.rowpart0[k], s1 = ws.rowpart1[k];
            lse_merge(m1, s1, M, S);
            ws.rowpart0[k] = m1; ws.rowpart1[k] = s1;
          }
        }
      }
    }
  }
  // merge row partials across strips (last CTA of this row block)
  if (arrive_last(ws.cnt_row + blockIdx.y, g.gx)) {
    double res = 0.0;
    for (int rt = blockIdx.y; rt < g.nrt; rt += g.gy) {
      for (int r = threadIdx.x; r < PINS_TR; r += PINS_TPB) {
        const int i = rt * PINS_TR + r;
        if (i >= m) break;
        double M = -INFINITY, S = 0.0;
        for (int x = 0; x < g.gx; ++x)
          lse_merge(M, S, __ldcg(ws.rowpart0 + (size_t)x * m + i), __ldcg(ws.rowpart1 + (size_t)x * m + i));
        double lse = M + log(S);
        double A = P::MIXED ? (double)p.Add[i].x + (double)p.Add[i].y : p.A64[i];
        double ai = p.a[i];
        res += fabs(exp(A + lse) - ai);
        F_out[i] = p.eta * (log(ai) + p.s - lse);
      }
    }
    double br = block_sum(res, sh_red);
    if (threadIdx.x == 0) ws.scal_row[blockIdx.y] = br;
  }
  if (arrive_last(ws.cnt_all, g.gx * g.gy)) {
    if (threadIdx.x == 0 && out_res) {
      double t = 0.0;
      for (int y = 0; y < g.gy; ++y) t += __ldcg(ws.scal_row + y);
      *out_res = t;
    }
  }
}

// ========================================================================= //
// 2. Sinkhorn column half-step (Alg. 2 warm-up, second update, new F):
//    G_j <- eta (log b_j - LSE_i (A_i - kappa C_ij)).
// ========================================================================= //
template <class P>
__global__ void __launch_bounds__(PINS_TPB)
k_col_lse(PassArgs p, TileGeom g, MergeWS ws, double* G_out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = p.m, n = p.n;
  __shared__ double shM[PINS_WARPS][PINS_TC];
  __shared__ double shS[PINS_WARPS][PINS_TC];
  float kh = p.kappa_dd.hi, kl = p.kappa_dd.lo;
  for (int ct = blockIdx.x; ct < g.nct; ct += g.gx) {
    int jj[PINS_CPL];
#pragma unroll
    for (int q = 0; q < PINS_CPL; ++q) jj[q] = ct * PINS_TC + lane + 32 * q;
    double cM[PINS_CPL], cS[PINS_CPL];
#pragma unroll
    for (int q = 0; q < PINS_CPL; ++q) { cM[q] = -INFINITY; cS[q] = 0.0; }
    for (int rt = blockIdx.y; rt < g.nrt; rt += g.gy) {
      if constexpr (!P::MIXED) {
        double v[PINS_RPT][PINS_CPL];
        double mx[PINS_CPL];
#pragma unroll
        for (int q = 0; q < PINS_CPL; ++q) mx[q] = -INFINITY;
#pragma unroll
        for (int t = 0; t < PINS_RPT; ++t) {
          const int i = rt * PINS_TR + warp + PINS_WARPS * t;
          double A = (i < m) ? P::row(p, i) : 0.0;
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
          float2 A = (i < m) ? P::row(p, i) : make_float2(0.f, 0.f);
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
          if (cM[q] == -INFINITY) { cM[q] = mx[q]; cS[q] = s; }
          else if ((double)mx[q] > cM[q]) { cS[q] = cS[q] * (double)exp2f((float)(cM[q] - mx[q]) * 1.4426950408889634f) + s; cM[q] = mx[q]; }
          else cS[q] += (double)(s * exp2f((float)(mx[q] - cM[q]) * 1.4426950408889634f));
        }
      }
    }
    // combine the 8 warps of this CTA per column
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PINS_CPL; ++q) { shM[warp][lane + 32 * q] = cM[q]; shS[warp][lane + 32 * q] = cS[q]; }
    __syncthreads();
    for (int c = threadIdx.x; c < PINS_TC; c += PINS_TPB) {
      double M = -INFINITY, S = 0.0;
      for (int w = 0; w < PINS_WARPS; ++w) lse_merge(M, S, shM[w][c], shS[w][c]);
      int j = ct * PINS_TC + c;
      if (j < n) {
        ws.colpart0[(size_t)blockIdx.y * n + j] = M;
        ws.colpart1[(size_t)blockIdx.y * n + j] = S;
      }
    }
    __syncthreads();
  }
  if (arrive_last(ws.cnt_col + blockIdx.x, g.gy)) {
    for (int ct = blockIdx.x; ct < g.nct; ct += g.gx) {
      for (int c = threadIdx.x; c < PINS_TC; c += PINS_TPB) {
        int j = ct * PINS_TC + c;
        if (j >= n) break;
        double M = -INFINITY, S = 0.0;
        for (int y = 0; y < g.gy; ++y)
          lse_merge(M, S, __ldcg(ws.colpart0 + (size_t)y * n + j), __ldcg(ws.colpart1 + (size_t)y * n + j));
        G_out[j] = p.eta * (log(p.b[j]) - (M + log(S)));
      }
    }
  }
}

// ========================================================================= //
// 3. Marginal pass (gradient after Eq. eppa-sub-dual) and the line-search trial
//    (Alg. 2 LineSearch, reading R7).  Per entry e = X~_ij = exp(z_ij).
//    TRIAL = false: r_i = sum_j e, c_j = sum_i e.
//    TRIAL = true : t_ij = Pt_i + Qt_j (= alpha (df_i + dg_j) / eta),
//                   e' = e (1 + expm1 t): r_i = sum_j e', c_j = sum_i e',
//                   d_i = sum_j e expm1(t)  (objective increase term).
//    Scalars (out[]): 0 residual ||r - a||_1 + ||c - b||_1, 1 sum X (of e or e'),
//                     2 max_ij z (of e or e'), 3 sum_i d_i (TRIAL).
// ========================================================================= //
struct TrialArgs {
  const double* Pt64; const double* Qt64;     // FP64 path
  const float2* Ptdd; const float2* Qtdd;     // mixed path
};

template <class P, bool TRIAL>
__global__ void __launch_bounds__(PINS_TPB)
k_marg(PassArgs p, TileGeom g, MergeWS ws, TrialArgs tr, double* r_out, double* c_out,
       double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = p.m, n = p.n;
  __shared__ double shC[PINS_WARPS][PINS_TC];
  __shared__ double sh_red[PINS_WARPS];
  __shared__ float2 s_tab[P::MIXED ? PINS_EXP_TABLE : 1];
  if constexpr (P::MIXED) {
    for (int q = threadIdx.x; q < PINS_EXP_TABLE; q += PINS_TPB) s_tab[q] = p.exp_table[q];
    __syncthreads();
  }
  float kh = p.kappa_dd.hi, kl = p.kappa_dd.lo;
  double zmax = -INFINITY;
  for (int ct = blockIdx.x; ct < g.nct; ct += g.gx) {
    const bool first = (ct == (int)blockIdx.x);
    int jj[PINS_CPL];
    typename P::Col cd[PINS_CPL];
    double Qd[PINS_CPL]; float2 Qf[PINS_CPL];
#pragma unroll
    for (int q = 0; q < PINS_CPL; ++q) {
      jj[q] = ct * PINS_TC + lane + 32 * q;
      int jc = jj[q] < n ? jj[q] : n - 1;
      cd[q] = P::col(p, jc);
      if constexpr (TRIAL) {
        if constexpr (P::MIXED) Qf[q] = tr.Qtdd[jc]; else Qd[q] = tr.Qt64[jc];
      }
    }
    double csum[PINS_CPL];
    dd cdd[PINS_CPL];
#pragma unroll
    for (int q = 0; q < PINS_CPL; ++q) { csum[q] = 0.0; cdd[q].hi = 0.f; cdd[q].lo = 0.f; }
    for (int rt = blockIdx.y; rt < g.nrt; rt += g.gy) {
#pragma unroll 2
      for (int t = 0; t < PINS_RPT; ++t) {
        const int i = rt * PINS_TR + warp + PINS_WARPS * t;
        if (i >= m) break;
        double rs = 0.0, ds = 0.0;
        if constexpr (!P::MIXED) {
          double A = P::row(p, i);
          double Pt = TRIAL ? tr.Pt64[i] : 0.0;
#pragma unroll
          for (int q = 0; q < PINS_CPL; ++q) {
            if (jj[q] >= n) continue;
            double z = A + fma(-p.kappa, P::cost(p, i, jj[q]), cd[q]);
            double e = exp(z);
            if constexpr (TRIAL) {
              double em1 = expm1(Pt + Qd[q]);
              double de = e * em1;
              ds += de;
              e = e + de;
              z = z + (Pt + Qd[q]);
            }
            zmax = fmax(zmax, z);
            rs += e;
            csum[q] += e;
          }
        } else {
          float2 A = P::row(p, i);
          float2 Pt = TRIAL ? tr.Ptdd[i] : make_float2(0.f, 0.f);
          dd racc; racc.hi = 0.f; racc.lo = 0.f;
          dd dacc; dacc.hi = 0.f; dacc.lo = 0.f;
#pragma unroll
          for (int q = 0; q < PINS_CPL; ++q) {
            if (jj[q] >= n) continue;
            float wh, wl, zh, zl;
            dd_w(cd[q], P::cost(p, i, jj[q]), kh, kl, wh, wl);
            dd_z(A, wh, wl, zh, zl);
            dd e = dd_exp(zh, zl, s_tab);
            if constexpr (TRIAL) {
              float th, tl; two_sum(Pt.x, Qf[q].x, th, tl);
              tl = __fadd_rn(tl, __fadd_rn(Pt.y, Qf[q].y));
              dd em1 = dd_expm1(th, tl, s_tab);
              dd de = dd_mul(e, em1);
              dd_acc(dacc, de.hi, de.lo);
              e = dd_add(e, de);
              zh = zh + th;
              zl = zl + tl;
            }
            // the FP32 value of z, as ranked by Sparsify (hi alone can be off by
            // |A| 2^-24 when A and B cancel)
            zmax = fmax(zmax, (double)__fadd_rn(zh, zl));
            dd_acc(racc, e.hi, e.lo);
            dd_acc(cdd[q], e.hi, e.lo);
          }
          rs = dd_to_double(racc);
          ds = dd_to_double(dacc);
        }
        rs = warp_sum(rs);
        if constexpr (TRIAL) ds = warp_sum(ds);
        if (lane == 0) {
          size_t k = (size_t)blockIdx.x * m + i;
          if (first) { ws.rowpart0[k] = rs; if (TRIAL) ws.rowpart1[k] = ds; }
          else { ws.rowpart0[k] += rs; if (TRIAL) ws.rowpart1[k] += ds; }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PINS_CPL; ++q)
      shC[warp][lane + 32 * q] = P::MIXED ? dd_to_double(cdd[q]) : csum[q];
    __syncthreads();
    for (int c = threadIdx.x; c < PINS_TC; c += PINS_TPB) {
      double S = 0.0;
      for (int w = 0; w < PINS_WARPS; ++w) S += shC[w][c];
      int j = ct * PINS_TC + c;
      if (j < n) ws.colpart0[(size_t)blockIdx.y * n + j] = S;
    }
    __syncthreads();
  }
  // per-CTA max of z goes to a scalar slot through the row-block partials
  double bmax = block_max(zmax, sh_red);
  if (threadIdx.x == 0) ws.scal_col[4 * (blockIdx.y * g.gx + blockIdx.x) + 3] = bmax;
  if (arrive_last(ws.cnt_row + blockIdx.y, g.gx)) {
    double res = 0.0, tot = 0.0, dsum = 0.0;
    for (int rt = blockIdx.y; rt < g.nrt; rt += g.gy) {
      for (int r = threadIdx.x; r < PINS_TR; r += PINS_TPB) {
        const int i = rt * PINS_TR + r;
        if (i >= m) break;
        double R = 0.0, D = 0.0;
        for (int x = 0; x < g.gx; ++x) {
          R += __ldcg(ws.rowpart0 + (size_t)x * m + i);
          if (TRIAL) D += __ldcg(ws.rowpart1 + (size_t)x * m + i);
        }
        r_out[i] = R;
        res += fabs(R - p.a[i]);
        tot += R;
        dsum += D;
      }
    }
    double b0 = block_sum(res, sh_red);
    double b1 = block_sum(tot, sh_red);
    double b2 = block_sum(dsum, sh_red);
    if (threadIdx.x == 0) {
      ws.scal_row[4 * blockIdx.y + 0] = b0;
      ws.scal_row[4 * blockIdx.y + 1] = b1;
      ws.scal_row[4 * blockIdx.y + 2] = b2;
    }
  }
  if (arrive_last(ws.cnt_col + blockIdx.x, g.gy)) {
    double res = 0.0;
    for (int ct = blockIdx.x; ct < g.nct; ct += g.gx) {
      for (int c = threadIdx.x; c < PINS_TC; c += PINS_TPB) {
        int j = ct * PINS_TC + c;
        if (j >= n) break;
        double S = 0.0;
        for (int y = 0; y < g.gy; ++y) S += __ldcg(ws.colpart0 + (size_t)y * n + j);
        c_out[j] = S;
        res += fabs(S - p.b[j]);
      }
    }
    double b0 = block_sum(res, sh_red);
    if (threadIdx.x == 0) ws.scal_col[4 * g.gx * g.gy + blockIdx.x] = b0;
  }
  if (arrive_last(ws.cnt_all, g.gx * g.gy)) {
    if (threadIdx.x == 0) {
      double res = 0.0, tot = 0.0, ds = 0.0, zm = -INFINITY;
      for (int y = 0; y < g.gy; ++y) {
        res += __ldcg(ws.scal_row + 4 * y + 0);
        tot += __ldcg(ws.scal_row + 4 * y + 1);
        ds += __ldcg(ws.scal_row + 4 * y + 2);
      }
      for (int x = 0; x < g.gx; ++x) res += __ldcg(ws.scal_col + 4 * g.gx * g.gy + x);
      for (int k = 0; k < g.gx * g.gy; ++k) zm = fmax(zm, __ldcg(ws.scal_col + 4 * k + 3));
      out[0] = res; out[1] = tot; out[2] = zm; out[3] = ds;
    }
  }
}

// ========================================================================= //
// 4. Certificate passes (reading R9 of the outer stop).
//    Column pass: c1_j = sum_i X~_ij xs_i  (xs_i = min(a_i / r_i, 1)),
//                 v_j  = min_i (C_ij - u_i) (u_i = F_i / s - eta).
//    Row pass:    rr_i = sum_j X~_ij xs_i ys_j, cr_i = sum_j C_ij X~_ij xs_i ys_j,
//                 cp_i = sum_j C_ij X~_ij, tc_i = sum_j C_ij ec_j,
//                 u2_i = min_j (C_ij - v_j).
//    Exact C_ij: FP64 policy evaluates it in FP64; the mixed policy uses
//    cscale * c32 in FP64 (the FP32 raw cost is the definition there).
// ========================================================================= //
struct CertArgs {
  const double* xs; const double* ys; const double* u; const double* v; const double* ec;
  double* c1; double* vout; double* rr; double* cr; double* cp; double* tc; double* u2;
};

template <class P>
__device__ __forceinline__ double exact_cost(const PassArgs& p, int i, int j) {
  if constexpr (P::MIXED) return p.cscale * (double)P::cost(p, i, j);
  else return P::cost(p, i, j);
}

template <class P>
__device__ __forceinline__ double entry_plan(const PassArgs& p, int i, int j,
                                             const float2* tab) {
  if constexpr (!P::MIXED) {
    return exp(P::row(p, i) + fma(-p.kappa, P::cost(p, i, j), P::col(p, j)));
  } else {
    float wh, wl, zh, zl;
    dd_w(P::col(p, j), P::cost(p, i, j), p.kappa_dd.hi, p.kappa_dd.lo, wh, wl);
    dd_z(P::row(p, i), wh, wl, zh, zl);
    dd e = dd_exp(zh, zl, tab);
    return dd_to_double(e);
  }
}

template <class P, bool COLPASS>
__global__ void __launch_bounds__(PINS_TPB)
k_cert(PassArgs p, TileGeom g, MergeWS ws, CertArgs ca) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = p.m, n = p.n;
  __shared__ double shA[PINS_WARPS][PINS_TC];
  __shared__ double shB[PINS_WARPS][PINS_TC];
  __shared__ float2 s_tab[P::MIXED ? PINS_EXP_TABLE : 1];
  if constexpr (P::MIXED) {
    for (int q = threadIdx.x; q < PINS_EXP_TABLE; q += PINS_TPB) s_tab[q] = p.exp_table[q];
    __syncthreads();
  }
  for (int ct = blockIdx.x; ct < g.nct; ct += g.gx) {
    const bool first = (ct == (int)blockIdx.x);
    double cs[PINS_CPL], cmin[PINS_CPL];
#pragma unroll
    for (int q = 0; q < PINS_CPL; ++q) { cs[q] = 0.0; cmin[q] = INFINITY; }
    for (int rt = blockIdx.y; rt < g.nrt; rt += g.gy) {
      for (int t = 0; t < PINS_RPT; ++t) {
        const int i = rt * PINS_TR + warp + PINS_WARPS * t;
        if (i >= m) break;
        double x_i = ca.xs[i];
        double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0, rmin = INFINITY;
#pragma unroll
        for (int q = 0; q < PINS_CPL; ++q) {
          const int j = ct * PINS_TC + lane + 32 * q;
          if (j >= n) continue;
          double e = entry_plan<P>(p, i, j, s_tab);
          double C = exact_cost<P>(p, i, j);
          if constexpr (COLPASS) {
            cs[q] += e * x_i;
            cmin[q] = fmin(cmin[q], C - ca.u[i]);
          } else {
            double ey = e * x_i * ca.ys[j];
            r0 += ey; r1 += C * ey; r2 += C * e; r3 += C * ca.ec[j];
            rmin = fmin(rmin, C - ca.v[j]);
          }
        }
        if constexpr (!COLPASS) {
          r0 = warp_sum(r0); r1 = warp_sum(r1); r2 = warp_sum(r2); r3 = warp_sum(r3);
          rmin = warp_mind(rmin);
          if (lane == 0) {
            size_t k = (size_t)blockIdx.x * m + i;
            if (first) { ws.rowpart0[k] = r0; ws.rowpart1[k] = r1; ws.rowpart2[k] = r2;
                         ws.rowpart3[k] = r3; ws.rowpart4[k] = rmin; }
            else { ws.rowpart0[k] += r0; ws.rowpart1[k] += r1; ws.rowpart2[k] += r2;
                   ws.rowpart3[k] += r3; ws.rowpart4[k] = fmin(ws.rowpart4[k], rmin); }
          }
        }
      }
    }
    if constexpr (COLPASS) {
      __syncthreads();
#pragma unroll
      for (int q = 0; q < PINS_CPL; ++q) { shA[warp][lane + 32 * q] = cs[q]; shB[warp][lane + 32 * q] = cmin[q]; }
      __syncthreads();
      for (int c = threadIdx.x; c < PINS_TC; c += PINS_TPB) {
        double S = 0.0, Mn = INFINITY;
        for (int w = 0; w < PINS_WARPS; ++w) { S += shA[w][c]; Mn = fmin(Mn, shB[w][c]); }
        int j = ct * PINS_TC + c;
        if (j < n) { ws.colpart0[(size_t)blockIdx.y * n + j] = S; ws.colpart1[(size_t)blockIdx.y * n + j] = Mn; }
      }
      __syncthreads();
    }
  }
  if constexpr (COLPASS) {
    if (arrive_last(ws.cnt_col + blockIdx.x, g.gy)) {
      for (int ct = blockIdx.x; ct < g.nct; ct += g.gx) {
        for (int c = threadIdx.x; c < PINS_TC; c += PINS_TPB) {
          int j = ct * PINS_TC + c;
          if (j >= n) break;
          double S = 0.0, Mn = INFINITY;
          for (int y = 0; y < g.gy; ++y) {
            S += __ldcg(ws.colpart0 + (size_t)y * n + j);
            Mn = fmin(Mn, __ldcg(ws.colpart1 + (size_t)y * n + j));
          }
          ca.c1[j] = S; ca.vout[j] = Mn;
        }
      }
    }
  } else {
    if (arrive_last(ws.cnt_row + blockIdx.y, g.gx)) {
      for (int rt = blockIdx.y; rt < g.nrt; rt += g.gy) {
        for (int r = threadIdx.x; r < PINS_TR; r += PINS_TPB) {
          const int i = rt * PINS_TR + r;
          if (i >= m) break;
          double s0 = 0, s1 = 0, s2 = 0, s3 = 0, mn = INFINITY;
          for (int x = 0; x < g.gx; ++x) {
            size_t k = (size_t)x * m + i;
            s0 += __ldcg(ws.rowpart0 + k); s1 += __ldcg(ws.rowpart1 + k);
            s2 += __ldcg(ws.rowpart2 + k); s3 += __ldcg(ws.rowpart3 + k);
            mn = fmin(mn, __ldcg(ws.rowpart4 + k));
          }
          ca.rr[i] = s0; ca.cr[i] = s1; ca.cp[i] = s2; ca.tc[i] = s3; ca.u2[i] = mn;
        }
      }
    }
  }
}

// ========================================================================= //
// 5. Sparsify passes (reading R5).  Ranking key: FP64 path k = (F_i + G_j) -
//    s (C_ij + eta) with no contraction; mixed path k = FP32 value of z_ij.
//    Window/binning: u = kref - k; bin = floor((u - lo) / width), bins < 0 are
//    above the window (definitely kept), bins >= NB below it.
// ========================================================================= //
#define PINS_HIST_NB 2048
#define PINS_CAND_CAP 8192

struct SparsifyState {      // device-resident, written by the select kernels
  double kref, lo, width;   // current window
  long long count_in;       // entries known to be above the window
  int level;
  int done;                 // 1: threshold bin fits the candidate buffer
  int need;                 // entries to take from the threshold bin
  int thr_bin;              // threshold bin
  unsigned int cand_count;  // candidates collected
  unsigned int coo_count;   // definitely-kept entries collected
  int overflow;             // error flag (candidate or COO overflow)
  int keep;                 // K
  double tau; long long tau_idx;  // final exact threshold (key, linear index)
};

template <class P>
__device__ __forceinline__ double rank_key(const PassArgs& p, int i, int j) {
  if constexpr (!P::MIXED) {
    double c = P::cost(p, i, j);
    return __dsub_rn(__dadd_rn(p.F[i], p.G[j]), __dmul_rn(p.s, __dadd_rn(c, p.eta)));
  } else {
    float wh, wl, zh, zl;
    dd_w(P::col(p, j), P::cost(p, i, j), p.kappa_dd.hi, p.kappa_dd.lo, wh, wl);
    dd_z(P::row(p, i), wh, wl, zh, zl);
    return (double)__fadd_rn(zh, zl);
  }
}

__device__ __forceinline__ int key_bin(double key, const SparsifyState& st) {
  double u = st.kref - key;
  double b = floor((u - st.lo) / st.width);
  if (b < 0.0) return -1;
  if (b >= (double)PINS_HIST_NB) return PINS_HIST_NB;
  return (int)b;
}

// histogram of the keys inside the current window (skipped once done)
template <class P>
__global__ void __launch_bounds__(PINS_TPB)
k_key_hist(PassArgs p, const SparsifyState* __restrict__ st_, unsigned int* hist) {
  __shared__ unsigned int sh[PINS_HIST_NB + 1];
  SparsifyState st = *st_;
  if (st.done) return;
  for (int q = threadIdx.x; q <= PINS_HIST_NB; q += PINS_TPB) sh[q] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int wpb = PINS_TPB / 32;
  for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < p.m; i += gridDim.x * wpb) {
    for (int j = lane; j < p.n; j += 32) {
      int b = key_bin(rank_key<P>(p, i, j), st);
      if (b >= 0 && b < PINS_HIST_NB) atomicAdd(&sh[b], 1u);
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < PINS_HIST_NB; q += PINS_TPB)
    if (sh[q]) atomicAdd(&hist[q], sh[q]);
}

// collect definitely-kept entries (COO) and threshold-bin candidates
template <class P>
__global__ void __launch_bounds__(PINS_TPB)
k_key_compact(PassArgs p, SparsifyState* st_, double* coo_key, long long* coo_idx,
              double* cand_key, long long* cand_idx, int coo_cap) {
  SparsifyState st = *st_;
  if (!st.done || st.overflow) return;
  const int lane = threadIdx.x & 31;
  const int wpb = PINS_TPB / 32;
  for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < p.m; i += gridDim.x * wpb)
  for (int j = lane; j < p.n; j += 32) {
    const long long e = (long long)i * p.n + j;
    double k = rank_key<P>(p, i, j);
    int b = key_bin(k, st);
    if (b < st.thr_bin) {
      unsigned int pos = atomicAdd(&st_->coo_count, 1u);
      if ((int)pos < coo_cap) { coo_key[pos] = k; coo_idx[pos] = e; }
      else st_->overflow = 1;
    } else if (b == st.thr_bin) {
      unsigned int pos = atomicAdd(&st_->cand_count, 1u);
      if (pos < PINS_CAND_CAP) { cand_key[pos] = k; cand_idx[pos] = e; }
      else st_->overflow = 1;
    }
  }
}

}  // namespace pins
