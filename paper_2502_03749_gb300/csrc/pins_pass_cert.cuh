// Certificate passes of the outer stopping test (reading R9).
//   Column pass: c1_j = sum_i X~_ij xs_i  (xs_i = min(a_i / r_i, 1)),
//                v_j  = min_i (C_ij - u_i) (u_i = F_i / s - eta),
//                vT_j = min_i (C_ij - uT_i) (uT: the support-tree dual).
//   Row pass:    rr_i = sum_j X~_ij xs_i ys_j, cr_i = sum_j C_ij X~_ij xs_i ys_j,
//                cp_i = sum_j C_ij X~_ij, tc_i = sum_j C_ij ec_j,
//                u2_i = min_j (C_ij - v_j), u2T_i = min_j (C_ij - vT_j).
// C_ij: the FP64 policy evaluates it in FP64; the mixed policy uses cscale * c32
// in FP64 (the FP32 raw cost is the definition of C there).  The entries are
// summed in FP64 (this pass runs once per certificate, not per step).
#pragma once

namespace pins {

struct CertArgs {
  const double* xs; const double* ys; const double* u; const double* v; const double* ec;
  double* c1; double* vout; double* rr; double* cr; double* cp; double* tc; double* u2;
  const double* uT; double* vTout; const double* vT; double* u2T;
};

template <class P>
__device__ __forceinline__ double exact_cost(const PassArgs& p, int i, int j) {
  if constexpr (P::MIXED) return p.cscale * (double)P::cost(p, i, j);
  else return P::cost(p, i, j);
}

template <class P>
__device__ __forceinline__ double entry_plan(const PassArgs& p, int i, int j, const float2* tab) {
  if constexpr (!P::MIXED) {
    return exp(P::row(p, i) + fma(-p.kappa, P::cost(p, i, j), P::col(p, j)));
  } else {
    float wh, wl, zh, zl;
    dd_w(P::col(p, j), P::cost(p, i, j), p.kappa_dd.hi, p.kappa_dd.lo, wh, wl);
    dd_z(P::row(p, i), wh, wl, zh, zl);
    return dd_to_double(dd_exp(zh, zl, tab));
  }
}

template <class P, bool COLPASS>
__global__ void __launch_bounds__(PINS_TPB)
k_cert(PassArgs p, TileGeom g, MergeWS ws, CertArgs ca) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = p.m, n = p.n;
  __shared__ double stg[2][PINS_STAGE];
  __shared__ float2 s_tab[P::MIXED ? PINS_EXP_TABLE : 1];
  if constexpr (P::MIXED) {
    for (int q = threadIdx.x; q < PINS_EXP_TABLE; q += PINS_TPB) s_tab[q] = p.exp_table[q];
    __syncthreads();
  }
  for (int ct = blockIdx.x; ct < g.nct; ct += g.gx) {
    const bool first = (ct == (int)blockIdx.x);
    double cs[PINS_CPL], cmin[PINS_CPL], cmin2[PINS_CPL];
#pragma unroll
    for (int q = 0; q < PINS_CPL; ++q) { cs[q] = 0.0; cmin[q] = INFINITY; cmin2[q] = INFINITY; }
    for (int rt = blockIdx.y; rt < g.nrt; rt += g.gy) {
      for (int t = 0; t < PINS_RPT; ++t) {
        const int i = rt * PINS_TR + warp + PINS_WARPS * t;
        if (i >= m) break;
        const double x_i = ca.xs[i];
        double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0, rmin = INFINITY, rmin2 = INFINITY;
#pragma unroll
        for (int q = 0; q < PINS_CPL; ++q) {
          const int j = ct * PINS_TC + lane + 32 * q;
          if (j >= n) continue;
          const double e = entry_plan<P>(p, i, j, s_tab);
          const double C = exact_cost<P>(p, i, j);
          if constexpr (COLPASS) {
            cs[q] += e * x_i;
            cmin[q] = fmin(cmin[q], C - ca.u[i]);
            cmin2[q] = fmin(cmin2[q], C - ca.uT[i]);
          } else {
            const double ey = e * x_i * ca.ys[j];
            r0 += ey; r1 += C * ey; r2 += C * e; r3 += C * ca.ec[j];
            rmin = fmin(rmin, C - ca.v[j]);
            rmin2 = fmin(rmin2, C - ca.vT[j]);
          }
        }
        if constexpr (!COLPASS) {
          r0 = warp_sum(r0); r1 = warp_sum(r1); r2 = warp_sum(r2); r3 = warp_sum(r3);
          rmin = warp_mind(rmin);
          rmin2 = warp_mind(rmin2);
          if (lane == 0) {
            const size_t k = (size_t)blockIdx.x * m + i;
            if (first) { ws.rowpart0[k] = r0; ws.rowpart1[k] = r1; ws.rowpart2[k] = r2;
                         ws.rowpart3[k] = r3; ws.rowpart4[k] = rmin; ws.rowpart5[k] = rmin2; }
            else { ws.rowpart0[k] += r0; ws.rowpart1[k] += r1; ws.rowpart2[k] += r2;
                   ws.rowpart3[k] += r3; ws.rowpart4[k] = fmin(ws.rowpart4[k], rmin);
                   ws.rowpart5[k] = fmin(ws.rowpart5[k], rmin2); }
          }
        }
      }
    }
    if constexpr (COLPASS) {
      __syncthreads();
#pragma unroll
      for (int q = 0; q < PINS_CPL; ++q) {
        stg[0][warp * PINS_TC + lane + 32 * q] = cs[q];
        stg[1][warp * PINS_TC + lane + 32 * q] = cmin[q];
      }
      __syncthreads();
      for (int c = threadIdx.x; c < PINS_TC; c += PINS_TPB) {
        double S = 0.0, Mn = INFINITY;
        for (int w = 0; w < PINS_WARPS; ++w) { S += stg[0][w * PINS_TC + c]; Mn = fmin(Mn, stg[1][w * PINS_TC + c]); }
        const int j = ct * PINS_TC + c;
        if (j < n) {
          ws.colpart0[(size_t)blockIdx.y * n + j] = S;
          ws.colpart1[(size_t)blockIdx.y * n + j] = Mn;
        }
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < PINS_CPL; ++q) stg[0][warp * PINS_TC + lane + 32 * q] = cmin2[q];
      __syncthreads();
      for (int c = threadIdx.x; c < PINS_TC; c += PINS_TPB) {
        double Mn = INFINITY;
        for (int w = 0; w < PINS_WARPS; ++w) Mn = fmin(Mn, stg[0][w * PINS_TC + c]);
        const int j = ct * PINS_TC + c;
        if (j < n) ws.colpart2[(size_t)blockIdx.y * n + j] = Mn;
      }
      __syncthreads();
    }
  }
  if constexpr (COLPASS) {
    if (arrive_last(ws.cnt_col + blockIdx.x, g.gy)) {
      for (int ct = blockIdx.x; ct < g.nct; ct += g.gx) {
        const int j0 = ct * PINS_TC;
        const int nc = min(PINS_TC, n - j0);
        double S = 0.0, Mn = INFINITY;
        for (int y0 = 0; y0 < g.gy; y0 += 16) {
          const int cnt = min(16, g.gy - y0);
          stage8(ws.colpart0 + (size_t)y0 * n + j0, n, cnt, PINS_TC, nc, stg[0]);
          stage8(ws.colpart1 + (size_t)y0 * n + j0, n, cnt, PINS_TC, nc, stg[1]);
          __syncthreads();
          if ((int)threadIdx.x < nc)
            for (int s = 0; s < cnt; ++s) {
              S += stg[0][s * PINS_TC + threadIdx.x];
              Mn = fmin(Mn, stg[1][s * PINS_TC + threadIdx.x]);
            }
          __syncthreads();
        }
        if ((int)threadIdx.x < nc) { ca.c1[j0 + threadIdx.x] = S; ca.vout[j0 + threadIdx.x] = Mn; }
        double Mn2 = INFINITY;
        for (int y0 = 0; y0 < g.gy; y0 += 16) {
          const int cnt = min(16, g.gy - y0);
          stage8(ws.colpart2 + (size_t)y0 * n + j0, n, cnt, PINS_TC, nc, stg[0]);
          __syncthreads();
          if ((int)threadIdx.x < nc)
            for (int s = 0; s < cnt; ++s) Mn2 = fmin(Mn2, stg[0][s * PINS_TC + threadIdx.x]);
          __syncthreads();
        }
        if ((int)threadIdx.x < nc) ca.vTout[j0 + threadIdx.x] = Mn2;
      }
    }
  } else {
    if (arrive_last(ws.cnt_row + blockIdx.y, g.gx)) {
      double* parts[6] = {ws.rowpart0, ws.rowpart1, ws.rowpart2, ws.rowpart3, ws.rowpart4,
                          ws.rowpart5};
      double* outs[6] = {ca.rr, ca.cr, ca.cp, ca.tc, ca.u2, ca.u2T};
      for (int rt = blockIdx.y; rt < g.nrt; rt += g.gy) {
        const int i0 = rt * PINS_TR;
        const int nr = min(PINS_TR, m - i0);
        for (int a = 0; a < 6; ++a) {
          stage8(parts[a] + i0, m, g.gx, PINS_TR, nr, stg[0]);
          __syncthreads();
          if ((int)threadIdx.x < nr) {
            double acc = (a >= 4) ? INFINITY : 0.0;
            for (int x = 0; x < g.gx; ++x) {
              const double v = stg[0][x * PINS_TR + threadIdx.x];
              acc = (a >= 4) ? fmin(acc, v) : acc + v;
            }
            outs[a][i0 + threadIdx.x] = acc;
          }
          __syncthreads();
        }
      }
    }
  }
}

}  // namespace pins
