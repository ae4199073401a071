// Marginal and line-search trial passes of the mixed policy (gradient after Eq.
// eppa-sub-dual; Algorithm 2 LineSearch, reading R7), in column segments.
//
// CTA (x, y) owns column segment x (PINS_MSEG columns) and the rows
// y*8 + w + t*8*gridDim.y (warp w).  For each row and half segment, lane l forms
// the exponents of 8 columns (2 chunks of 4 consecutive columns, 16-byte cost
// loads); the entries whose X~ is at least e^-87 (the others add nothing to any
// sum) are compacted into a per-warp list, and the double-float exp then runs
// on full warps over the list.  Column sums accumulate per warp in shared
// memory (a column appears once per row, so no two lanes share a slot), row
// sums in registers with one warp reduction per row.  B_j (and the trial
// increments Q_j) of the segment and the 2^(q/1024) table are staged in shared
// memory.  Partials are merged by the last CTA to arrive, in a fixed order, so
// results do not depend on scheduling.
//
// Per entry e = X~_ij = exp(z_ij) (double-float exp):
//   TRIAL = false: r_i = sum_j e, c_j = sum_i e.
//   TRIAL = true : t_ij = Pt_i + Qt_j (= alpha (df_i + dg_j) / eta),
//                  e' = exp(z + t): r_i = sum_j e', c_j = sum_i e',
//                  d_i = sum_j e (expm1(t) - t) in FP32 (see pins_pass_marg.cuh).
// Scalars (out[]): 0 residual ||r - a||_1 + ||c - b||_1, 1 sum X, 2 max_ij z,
// 3 sum_i d_i (TRIAL).
#pragma once

namespace pins {

#define PINS_MSEG 512
#define PINS_MHALF 256     // columns of a segment compacted at a time
// shared memory: exp table, B and Q of the segment, per-warp column sums
// (PINS_WARPS x PINS_MSEG double-float), per-warp compaction lists
#define PINS_MSEG_SMEM (sizeof(float2) * (PINS_EXP_TABLE + 2 * PINS_MSEG + PINS_WARPS * PINS_MSEG) + \
                        (sizeof(float2) + sizeof(int)) * PINS_WARPS * PINS_MHALF)

template <class P, bool TRIAL>
__global__ void __launch_bounds__(PINS_TPB)
k_marg_mx(PassArgs p, MergeWS ws, TrialArgs tr, double* r_out, double* c_out, double* out) {
  extern __shared__ float2 msm[];
  float2* s_tab = msm;
  float2* sB = s_tab + PINS_EXP_TABLE;
  float2* sQ = sB + PINS_MSEG;
  float2* cacc = sQ + PINS_MSEG;                            // [warp][column] sums
  float2* lz = cacc + PINS_WARPS * PINS_MSEG;                // [warp][slot]
  int* lc = reinterpret_cast<int*>(lz + PINS_WARPS * PINS_MHALF);
  __shared__ double sh_red[PINS_WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned int lt = (1u << lane) - 1u;
  const int m = p.m, n = p.n;
  const int x = blockIdx.x, y = blockIdx.y, SX = gridDim.x, GY = gridDim.y;
  const int j0 = x * PINS_MSEG, j1 = min(n, j0 + PINS_MSEG);
  for (int q = threadIdx.x; q < PINS_EXP_TABLE; q += PINS_TPB) s_tab[q] = p.exp_table[q];
  for (int j = j0 + threadIdx.x; j < j1; j += PINS_TPB) {
    sB[j - j0] = p.Bdd[j];
    if constexpr (TRIAL) sQ[j - j0] = ddv_mul(split_f64(tr.dir[m + j], 0), tr.scale);
  }
  for (int q = threadIdx.x; q < PINS_WARPS * PINS_MSEG; q += PINS_TPB) cacc[q] = make_float2(0.f, 0.f);
  __syncthreads();
  float2* wacc = cacc + warp * PINS_MSEG;
  float2* wlz = lz + warp * PINS_MHALF;
  int* wlc = lc + warp * PINS_MHALF;
  const float kh = p.kappa_dd.hi, kl = p.kappa_dd.lo;
  float zmaxf = -INFINITY;
  for (int i = y * PINS_WARPS + warp; i < m; i += GY * PINS_WARPS) {
    const float2 A = p.Add[i];
    const float2 Pt = TRIAL ? ddv_mul(split_f64(tr.dir[i], 0), tr.scale) : make_float2(0.f, 0.f);
    dd racc; racc.hi = 0.f; racc.lo = 0.f;
    float dfs = 0.f;
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      // 1. exponents of the half segment; entries whose X~ (at either point) is
      //    at least e^-87 go to the warp's list, so the double-float exp below
      //    runs on full warps
      int cnt = 0;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const int col0 = 4 * lane + 128 * (2 * hf + kk);
        const int jb = j0 + col0;
        float c[4];
        cost4<P>(p, i, jb, j1, c);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = jb + q;
          bool keep = false;
          float zh = 0.f, zl = 0.f;
          if (j < j1) {
            // FP32 estimate of z from the leading parts; its error is below a
            // few ulps of the largest term, so with the bound `lim` an entry
            // estimated below it is below e^-87 at the evaluated point(s) and
            // skips the double-float exponent: the kept set is exactly that of
            // the exact test
            const float2 Bj = sB[j - j0];
            const float kc = __fmul_rn(kh, c[q]);
            const float est = __fadd_rn(A.x, __fsub_rn(Bj.x, kc));
            const float lim = __fmaf_rn(-2.5e-7f, fabsf(A.x) + fabsf(Bj.x) + kc, -88.0f);
            float zf = est;
            float t1 = 0.f;
            if constexpr (TRIAL) {
              t1 = __fadd_rn(Pt.x, sQ[j - j0].x);
              keep = (est > lim) || (__fadd_rn(est, t1) > lim - 2.5e-7f * fabsf(t1));
              zf = __fadd_rn(est, t1);
            } else {
              keep = est > lim;
            }
            if (keep) {
              float wh, wl;
              dd_w(Bj, c[q], kh, kl, wh, wl);
              dd_z(A, wh, wl, zh, zl);
              zf = __fadd_rn(zh, zl);
              if constexpr (TRIAL) {
                // FP32 estimate of the trial point's exponent: it only places the
                // e^-87 skip threshold and the sparsify window; the listed
                // entries get z + t in double-float below
                const float z1 = __fadd_rn(zf, t1);
                keep = (zf > -87.0f) || (z1 > -87.0f);
                zf = z1;
              } else {
                keep = zf > -87.0f;
              }
            }
            zmaxf = fmaxf(zmaxf, zf);
          }
          const unsigned int bal = __ballot_sync(0xffffffffu, keep);
          if (keep) {
            const int pos = cnt + __popc(bal & lt);
            wlz[pos] = make_float2(zh, zl);
            wlc[pos] = col0 + q;
          }
          cnt += __popc(bal);
        }
      }
      __syncwarp();
      // 2. the listed entries, 32 at a time
      for (int l = lane; l < cnt; l += 32) {
        const float2 zz = wlz[l];
        const int col = wlc[l];
        float zh = zz.x, zl = zz.y;
        float z0 = 0.f, tf = 0.f;
        if constexpr (TRIAL) {
          // t = Pt_i + Qt_j and the trial point z + t in double-float
          const float2 Q = sQ[col];
          float th, tl; two_sum(Pt.x, Q.x, th, tl);
          tl = __fadd_rn(tl, __fadd_rn(Pt.y, Q.y));
          z0 = __fadd_rn(zh, zl);
          tf = __fadd_rn(th, tl);
          float sh, se; two_sum(zh, th, sh, se);
          se = __fadd_rn(se, __fadd_rn(zl, tl));
          fast_two_sum(sh, se, zh, zl);
        }
        const dd e = dd_exp(zh, zl, s_tab);
        dd_acc(racc, e.hi, e.lo);
        const float2 o = wacc[col];
        dd cc; cc.hi = o.x; cc.lo = o.y;
        dd_acc(cc, e.hi, e.lo);
        wacc[col] = make_float2(cc.hi, cc.lo);
        if constexpr (TRIAL) dfs = __fadd_rn(dfs, trial_term(z0, tf, e.hi));
      }
      __syncwarp();
    }
    racc = warp_dd_sum(racc);
    dd dacc; dacc.hi = dfs; dacc.lo = 0.f;
    if constexpr (TRIAL) dacc = warp_dd_sum(dacc);
    if (lane == 0) {
      store_f2(ws.rowpart0 + (size_t)x * m + i, racc.hi, racc.lo);
      if constexpr (TRIAL) store_f2(ws.rowpart1 + (size_t)x * m + i, dacc.hi, dacc.lo);
    }
  }
  // column partials of this CTA: the 8 warps merged in warp order
  __syncthreads();
  for (int cidx = threadIdx.x; cidx < PINS_MSEG; cidx += PINS_TPB) {
    const int j = j0 + cidx;
    if (j >= n) continue;
    dd acc; acc.hi = 0.f; acc.lo = 0.f;
#pragma unroll
    for (int w = 0; w < PINS_WARPS; ++w) {
      const float2 o = cacc[w * PINS_MSEG + cidx];
      acc = dd_add(acc, dd{o.x, o.y});
    }
    store_f2(ws.colpart0 + (size_t)y * n + j, acc.hi, acc.lo);
  }
  const double bmax = block_max((double)zmaxf, sh_red);
  if (threadIdx.x == 0) ws.scal_col[4 * (y * SX + x) + 3] = bmax;
  // rows of this row group, merged over the SX segments in segment order
  if (arrive_last(ws.cnt_row + y, SX)) {
    double res = 0.0, tot = 0.0, dsum = 0.0;
    const int per = PINS_WARPS * ((m + GY * PINS_WARPS - 1) / (GY * PINS_WARPS));
    for (int k = threadIdx.x; k < per; k += PINS_TPB) {
      const int i = y * PINS_WARPS + (k % PINS_WARPS) + (k / PINS_WARPS) * GY * PINS_WARPS;
      if (i >= m) continue;
      dd ar; ar.hi = 0.f; ar.lo = 0.f;
      dd ad; ad.hi = 0.f; ad.lo = 0.f;
      for (int xs = 0; xs < SX; ++xs) {
        const float2 o = load_f2_cg(ws.rowpart0 + (size_t)xs * m + i);
        ar = dd_add(ar, dd{o.x, o.y});
        if constexpr (TRIAL) {
          const float2 o1 = load_f2_cg(ws.rowpart1 + (size_t)xs * m + i);
          ad = dd_add(ad, dd{o1.x, o1.y});
        }
      }
      const double R = dd_to_double(ar);
      r_out[i] = R;
      res += fabs(R - p.a[i]);
      tot += R;
      dsum += dd_to_double(ad);
    }
    const double b0 = block_sum(res, sh_red);
    const double b1 = block_sum(tot, sh_red);
    const double b2 = block_sum(dsum, sh_red);
    const double zv = ((int)threadIdx.x < SX) ? __ldcg(ws.scal_col + 4 * (y * SX + threadIdx.x) + 3)
                                             : -INFINITY;
    const double b3 = block_max(zv, sh_red);
    if (threadIdx.x == 0) {
      ws.scal_row[4 * y + 0] = b0;
      ws.scal_row[4 * y + 1] = b1;
      ws.scal_row[4 * y + 2] = b2;
      ws.scal_row[4 * y + 3] = b3;
    }
  }
  // columns of this segment, merged over the GY row groups in group order
  if (arrive_last(ws.cnt_col + x, GY)) {
    double res = 0.0;
    for (int cidx = threadIdx.x; cidx < PINS_MSEG; cidx += PINS_TPB) {
      const int j = j0 + cidx;
      if (j >= n) continue;
      dd acc; acc.hi = 0.f; acc.lo = 0.f;
      for (int yb = 0; yb < GY; ++yb) {
        const float2 o = load_f2_cg(ws.colpart0 + (size_t)yb * n + j);
        acc = dd_add(acc, dd{o.x, o.y});
      }
      const double S = dd_to_double(acc);
      c_out[j] = S;
      res += fabs(S - p.b[j]);
    }
    const double b0 = block_sum(res, sh_red);
    if (threadIdx.x == 0) ws.scal_col[4 * PINS_GX_MAX * PINS_GY_MAX + x] = b0;
  }
  // the last CTA overall: scalars
  if (arrive_last(ws.cnt_all, SX * GY)) {
    const int t = threadIdx.x;
    const bool ry = t < GY, cx = t < SX;
    const double r0 = ry ? __ldcg(ws.scal_row + 4 * t + 0) : 0.0;
    const double r1 = ry ? __ldcg(ws.scal_row + 4 * t + 1) : 0.0;
    const double r2 = ry ? __ldcg(ws.scal_row + 4 * t + 2) : 0.0;
    const double r3 = ry ? __ldcg(ws.scal_row + 4 * t + 3) : -INFINITY;
    const double c0 = cx ? __ldcg(ws.scal_col + 4 * PINS_GX_MAX * PINS_GY_MAX + t) : 0.0;
    const double res = block_sum(r0, sh_red) + block_sum(c0, sh_red);
    const double tot = block_sum(r1, sh_red);
    const double ds = block_sum(r2, sh_red);
    const double zm = block_max(r3, sh_red);
    if (t == 0) { out[0] = res; out[1] = tot; out[2] = zm; out[3] = ds; }
  }
}

}  // namespace pins
