// Marginal pass (gradient after Eq. eppa-sub-dual) and the line-search trial
// pass (Algorithm 2 LineSearch, reading R7).  Per entry e = X~_ij = exp(z_ij).
//   TRIAL = false: r_i = sum_j e, c_j = sum_i e.
//   TRIAL = true : t_ij = Pt_i + Qt_j (= alpha (df_i + dg_j) / eta),
//                  e' = exp(z + t): r_i = sum_j e', c_j = sum_i e', and the
//                  objective increase term d_i:
//                  FP64 policy  d_i = sum_j e expm1(t)          (as the oracle)
//                  mixed policy d_i = sum_j e (expm1(t) - t)    (FP32, >= 0)
//   The two give the same increase: P(x + alpha d) - P(x)
//     = alpha (<a,df> + <b,dg>) - eta sum e expm1(t)
//     = alpha (<a - r, df> + <b - c, dg>) - eta sum e (expm1(t) - t),
//   since sum_ij e t_ij = (alpha / eta)(<r, df> + <c, dg>).  The second form has
//   no cancellation between its terms, so FP32 is enough for the sum.
// Scalars (out[]): 0 residual ||r - a||_1 + ||c - b||_1, 1 sum X (of e or e'),
//                  2 max_ij z (of e or e'), 3 sum_i d_i (TRIAL).
#pragma once

namespace pins {

struct TrialArgs {
  const double* Pt64; const double* Qt64;     // FP64 path: alpha df / eta, alpha dg / eta
  const double* dir;                          // mixed path: (df; dg), m + n
  float2 scale;                               // mixed path: alpha / eta as a pair
};

template <class P, bool TRIAL>
__global__ void __launch_bounds__(PINS_TPB)
k_marg(PassArgs p, TileGeom g, MergeWS ws, TrialArgs tr, double* r_out, double* c_out,
       double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = p.m, n = p.n;
  __shared__ double stg[2][PINS_STAGE];
  __shared__ double sh_red[PINS_WARPS];
  __shared__ float2 s_tab[P::MIXED ? PINS_EXP_TABLE : 1];
  if constexpr (P::MIXED) {
    for (int q = threadIdx.x; q < PINS_EXP_TABLE; q += PINS_TPB) s_tab[q] = p.exp_table[q];
    __syncthreads();
  }
  const float kh = p.kappa_dd.hi, kl = p.kappa_dd.lo;
  double zmax = -INFINITY;
  float zmaxf = -INFINITY;
  for (int ct = blockIdx.x; ct < g.nct; ct += g.gx) {
    const bool first = (ct == (int)blockIdx.x);
    int jj[PINS_CPL];
    typename P::Col cd[PINS_CPL];
    double Qd[PINS_CPL]; float2 Qf[PINS_CPL];
#pragma unroll
    for (int q = 0; q < PINS_CPL; ++q) {
      jj[q] = ct * PINS_TC + lane + 32 * q;
      const int jc = jj[q] < n ? jj[q] : n - 1;
      cd[q] = P::col(p, jc);
      if constexpr (TRIAL) {
        if constexpr (P::MIXED) Qf[q] = ddv_mul(split_f64(tr.dir[m + jc], 0), tr.scale);
        else Qd[q] = tr.Qt64[jc];
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
        const size_t k = (size_t)blockIdx.x * m + i;
        if constexpr (!P::MIXED) {
          const double A = P::row(p, i);
          const double Pt = TRIAL ? tr.Pt64[i] : 0.0;
          double rs = 0.0, ds = 0.0;
#pragma unroll
          for (int q = 0; q < PINS_CPL; ++q) {
            if (jj[q] >= n) continue;
            double z = A + fma(-p.kappa, P::cost(p, i, jj[q]), cd[q]);
            double e = exp(z);
            if constexpr (TRIAL) {
              const double em1 = expm1(Pt + Qd[q]);
              const double de = e * em1;
              ds += de;
              e = e + de;
              z = z + (Pt + Qd[q]);
            }
            zmax = fmax(zmax, z);
            rs += e;
            csum[q] += e;
          }
          rs = warp_sum(rs);
          if constexpr (TRIAL) ds = warp_sum(ds);
          if (lane == 0) {
            if (first) { ws.rowpart0[k] = rs; if (TRIAL) ws.rowpart1[k] = ds; }
            else { ws.rowpart0[k] += rs; if (TRIAL) ws.rowpart1[k] += ds; }
          }
        } else {
          const float2 A = P::row(p, i);
          const float2 Pt = TRIAL ? ddv_mul(split_f64(tr.dir[i], 0), tr.scale) : make_float2(0.f, 0.f);
          dd racc; racc.hi = 0.f; racc.lo = 0.f;
          float dfs = 0.f;
#pragma unroll
          for (int q = 0; q < PINS_CPL; ++q) {
            if (jj[q] >= n) continue;
            float wh, wl, zh, zl;
            dd_w(cd[q], P::cost(p, i, jj[q]), kh, kl, wh, wl);
            dd_z(A, wh, wl, zh, zl);
            if constexpr (TRIAL) {
              float th, tl; two_sum(Pt.x, Qf[q].x, th, tl);
              tl = __fadd_rn(tl, __fadd_rn(Pt.y, Qf[q].y));
              const float z0 = __fadd_rn(zh, zl);
              const float tf = __fadd_rn(th, tl);
              // trial point z + t in double-float
              float sh, se; two_sum(zh, th, sh, se);
              se = __fadd_rn(se, __fadd_rn(zl, tl));
              fast_two_sum(sh, se, zh, zl);
              // the FP32 value of z, as ranked by Sparsify (hi alone can be off by
              // |A| 2^-24 when A and B cancel)
              zmaxf = fmaxf(zmaxf, __fadd_rn(zh, zl));
              // X~ below e^-87 at both points: no term of any sum changes
              if (!(z0 > -87.0f) && !(zh > -87.0f)) continue;
              const dd e = dd_exp(zh, zl, s_tab);
              dd_acc(racc, e.hi, e.lo);
              dd_acc(cdd[q], e.hi, e.lo);
              dfs = __fadd_rn(dfs, trial_term(z0, tf, e.hi));
              continue;
            } else {
              zmaxf = fmaxf(zmaxf, __fadd_rn(zh, zl));
              if (!(zh > -87.0f)) continue;   // dd_exp gives 0: nothing to add
            }
            const dd e = dd_exp(zh, zl, s_tab);
            dd_acc(racc, e.hi, e.lo);
            dd_acc(cdd[q], e.hi, e.lo);
          }
          // row partial reduced across the warp in double-float, kept raw
          racc = warp_dd_sum(racc);
          dd dacc; dacc.hi = dfs; dacc.lo = 0.f;
          if constexpr (TRIAL) dacc = warp_dd_sum(dacc);
          if (lane == 0) {
            if (!first) {
              const float2 o = load_f2(ws.rowpart0 + k);
              racc = dd_add(racc, dd{o.x, o.y});
              if constexpr (TRIAL) {
                const float2 o1 = load_f2(ws.rowpart1 + k);
                dacc = dd_add(dacc, dd{o1.x, o1.y});
              }
            }
            store_f2(ws.rowpart0 + k, racc.hi, racc.lo);
            if constexpr (TRIAL) store_f2(ws.rowpart1 + k, dacc.hi, dacc.lo);
          }
        }
      }
    }
    // combine the 8 warps of this CTA per column
    __syncthreads();
    if constexpr (P::MIXED) {
#pragma unroll
      for (int q = 0; q < PINS_CPL; ++q) {
        float2 v = make_float2(cdd[q].hi, cdd[q].lo);
        stg[0][warp * PINS_TC + lane + 32 * q] = *reinterpret_cast<double*>(&v);
      }
      __syncthreads();
      for (int c = threadIdx.x; c < PINS_TC; c += PINS_TPB) {
        dd acc; acc.hi = 0.f; acc.lo = 0.f;
        for (int w = 0; w < PINS_WARPS; ++w) {
          const float2 o = as_f2(stg[0][w * PINS_TC + c]);
          acc = dd_add(acc, dd{o.x, o.y});
        }
        const int j = ct * PINS_TC + c;
        if (j < n) store_f2(ws.colpart0 + (size_t)blockIdx.y * n + j, acc.hi, acc.lo);
      }
    } else {
#pragma unroll
      for (int q = 0; q < PINS_CPL; ++q) stg[0][warp * PINS_TC + lane + 32 * q] = csum[q];
      __syncthreads();
      for (int c = threadIdx.x; c < PINS_TC; c += PINS_TPB) {
        double S = 0.0;
        for (int w = 0; w < PINS_WARPS; ++w) S += stg[0][w * PINS_TC + c];
        const int j = ct * PINS_TC + c;
        if (j < n) ws.colpart0[(size_t)blockIdx.y * n + j] = S;
      }
    }
    __syncthreads();
  }
  // per-CTA max of z
  if constexpr (P::MIXED) zmax = (double)zmaxf;
  const double bmax = block_max(zmax, sh_red);
  if (threadIdx.x == 0) ws.scal_col[4 * (blockIdx.y * g.gx + blockIdx.x) + 3] = bmax;
  // rows of this row block: staged merge over the strips
  if (arrive_last(ws.cnt_row + blockIdx.y, g.gx)) {
    double res = 0.0, tot = 0.0, dsum = 0.0;
    for (int rt = blockIdx.y; rt < g.nrt; rt += g.gy) {
      const int i0 = rt * PINS_TR;
      const int nr = min(PINS_TR, m - i0);
      stage8(ws.rowpart0 + i0, m, g.gx, PINS_TR, nr, stg[0]);
      if (TRIAL) stage8(ws.rowpart1 + i0, m, g.gx, PINS_TR, nr, stg[1]);
      __syncthreads();
      if ((int)threadIdx.x < nr) {
        const int i = i0 + threadIdx.x;
        double R = 0.0, D = 0.0;
        if constexpr (P::MIXED) {
          dd ar; ar.hi = 0.f; ar.lo = 0.f;
          dd ad; ad.hi = 0.f; ad.lo = 0.f;
          for (int x = 0; x < g.gx; ++x) {
            const float2 o = as_f2(stg[0][x * PINS_TR + threadIdx.x]);
            ar = dd_add(ar, dd{o.x, o.y});
            if (TRIAL) {
              const float2 o1 = as_f2(stg[1][x * PINS_TR + threadIdx.x]);
              ad = dd_add(ad, dd{o1.x, o1.y});
            }
          }
          R = dd_to_double(ar);
          D = dd_to_double(ad);
        } else {
          for (int x = 0; x < g.gx; ++x) {
            R += stg[0][x * PINS_TR + threadIdx.x];
            if (TRIAL) D += stg[1][x * PINS_TR + threadIdx.x];
          }
        }
        r_out[i] = R;
        res += fabs(R - p.a[i]);
        tot += R;
        dsum += D;
      }
      __syncthreads();
    }
    const double b0 = block_sum(res, sh_red);
    const double b1 = block_sum(tot, sh_red);
    const double b2 = block_sum(dsum, sh_red);
    const double zv = ((int)threadIdx.x < g.gx)
                          ? __ldcg(ws.scal_col + 4 * (blockIdx.y * g.gx + threadIdx.x) + 3)
                          : -INFINITY;
    const double b3 = block_max(zv, sh_red);
    if (threadIdx.x == 0) {
      ws.scal_row[4 * blockIdx.y + 0] = b0;
      ws.scal_row[4 * blockIdx.y + 1] = b1;
      ws.scal_row[4 * blockIdx.y + 2] = b2;
      ws.scal_row[4 * blockIdx.y + 3] = b3;
    }
  }
  // columns of this strip: staged merge over the row blocks, 16 at a time
  if (arrive_last(ws.cnt_col + blockIdx.x, g.gy)) {
    double res = 0.0;
    for (int ct = blockIdx.x; ct < g.nct; ct += g.gx) {
      const int j0 = ct * PINS_TC;
      const int nc = min(PINS_TC, n - j0);
      dd acc; acc.hi = 0.f; acc.lo = 0.f;
      double S = 0.0;
      for (int y0 = 0; y0 < g.gy; y0 += 16) {
        const int cnt = min(16, g.gy - y0);
        stage8(ws.colpart0 + (size_t)y0 * n + j0, n, cnt, PINS_TC, nc, stg[0]);
        __syncthreads();
        if ((int)threadIdx.x < nc) {
          for (int s = 0; s < cnt; ++s) {
            if constexpr (P::MIXED) {
              const float2 o = as_f2(stg[0][s * PINS_TC + threadIdx.x]);
              acc = dd_add(acc, dd{o.x, o.y});
            } else {
              S += stg[0][s * PINS_TC + threadIdx.x];
            }
          }
        }
        __syncthreads();
      }
      if ((int)threadIdx.x < nc) {
        if constexpr (P::MIXED) S = dd_to_double(acc);
        const int j = j0 + threadIdx.x;
        c_out[j] = S;
        res += fabs(S - p.b[j]);
      }
    }
    const double b0 = block_sum(res, sh_red);
    if (threadIdx.x == 0) ws.scal_col[4 * g.gx * g.gy + blockIdx.x] = b0;
  }
  // the last CTA overall: scalars, every thread loading one partial
  if (arrive_last(ws.cnt_all, g.gx * g.gy)) {
    const int t = threadIdx.x;
    const bool ry = t < g.gy, cx = t < g.gx;
    const double r0 = ry ? __ldcg(ws.scal_row + 4 * t + 0) : 0.0;
    const double r1 = ry ? __ldcg(ws.scal_row + 4 * t + 1) : 0.0;
    const double r2 = ry ? __ldcg(ws.scal_row + 4 * t + 2) : 0.0;
    const double r3 = ry ? __ldcg(ws.scal_row + 4 * t + 3) : -INFINITY;
    const double c0 = cx ? __ldcg(ws.scal_col + 4 * g.gx * g.gy + t) : 0.0;
    const double res = block_sum(r0, sh_red) + block_sum(c0, sh_red);
    const double tot = block_sum(r1, sh_red);
    const double ds = block_sum(r2, sh_red);
    const double zm = block_max(r3, sh_red);
    if (t == 0) { out[0] = res; out[1] = tot; out[2] = zm; out[3] = ds; }
  }
}

}  // namespace pins
