// Sinkhorn warm-up half-steps of the mixed policy (Algorithm 2 warm-up loop;
// Algorithm 1 in log form), streamed with an online log-sum-exp in base 2.
//
// The passes form log2(e) A_i, log2(e) B_j (from the FP64 potentials, split by
// integer operations) and log2(e) kappa as double-float pairs, so
// w = V - kappa C_ij is formed in double-float directly in log2 units
// and each entry costs one FP32 ex2 (flush-to-zero: a term below 2^-126 of the
// running maximum is dropped).  Each thread keeps a running (M, S) with
// S = sum 2^(w - M) and updates it four entries at a time: M' = max(M, the
// four w), S = S 2^(M - M') + sum 2^((w_hi - M') + w_lo).  No branch, no tile
// of w held in registers, no per-tile maximum pass.
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

__device__ __forceinline__ float ex2_ftz(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// four entries into a running base-2 (M, S); every wh finite
__device__ __forceinline__ void lse2_chunk(float& M, float& S, const float wh[4],
                                           const float wl[4]) {
  const float Mn = fmaxf(M, fmaxf(fmaxf(wh[0], wh[1]), fmaxf(wh[2], wh[3])));
  float t = __fmul_rn(S, ex2_ftz(__fsub_rn(M, Mn)));    // M = -inf: 2^-inf = 0
#pragma unroll
  for (int q = 0; q < 4; ++q) t = __fadd_rn(t, ex2_ftz(__fadd_rn(__fsub_rn(wh[q], Mn), wl[q])));
  S = t;
  M = Mn;
}
// one entry (tails)
__device__ __forceinline__ void lse2_one(float& M, float& S, float wh, float wl) {
  const float Mn = fmaxf(M, wh);
  S = __fadd_rn(__fmul_rn(S, ex2_ftz(__fsub_rn(M, Mn))), ex2_ftz(__fadd_rn(__fsub_rn(wh, Mn), wl)));
  M = Mn;
}
// base-2 LSE pair merge
__device__ __forceinline__ void lse2_merge(float& m1, float& s1, float m2, float s2) {
  if (m2 == -INFINITY) return;
  if (m1 == -INFINITY) { m1 = m2; s1 = s2; return; }
  const float mn = fmaxf(m1, m2);
  s1 = __fadd_rn(__fmul_rn(s1, ex2_ftz(__fsub_rn(m1, mn))), __fmul_rn(s2, ex2_ftz(__fsub_rn(m2, mn))));
  m1 = mn;
}

// log2(e) A_i = (F_i / eta - s) log2(e) as a pair, from the FP64 F_i
__device__ __forceinline__ float2 a2_of(const PassArgs& p, int i) {
  const float2 f = ddv_mul(split_f64(p.F[i], 0), p.l2e_eta);
  return ddv_add(f, make_float2(-p.s_l2e.x, -p.s_l2e.y));
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
  } else if constexpr (std::is_same<P, PolMixed<COST_GRID>>::value) {
    // grid cost: one division per row and per chunk; consecutive columns step
    // along the grid row (integers exact in FP32)
    const int s2 = p.cost.s2;
    const int i1 = i / s2, i2 = i - i1 * s2;
    int j1 = j / s2, j2 = j - j1 * s2;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int d1 = i1 - j1, d2 = i2 - j2;
      c[q] = (j + q < jend) ? (float)(d1 * d1 + d2 * d2) : 0.f;
      if (++j2 == s2) { j2 = 0; ++j1; }
    }
  } else if constexpr (std::is_same<P, PolMixed<COST_POINTS>>::value) {
    if (p.cost.d == 2) {      // planar points: the row point once, 8-byte column points
      const float2 xi = __ldg(reinterpret_cast<const float2*>(p.cost.xf) + i);
      const float2* yv = reinterpret_cast<const float2*>(p.cost.yf);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (j + q < jend) {
          const float2 yj = __ldg(yv + j + q);
          const float d0 = xi.x - yj.x, d1 = xi.y - yj.y;
          c[q] = __fmaf_rn(d1, d1, d0 * d0);
        } else {
          c[q] = 0.f;
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) c[q] = (j + q < jend) ? P::cost(p, i, j + q) : 0.f;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) c[q] = (j + q < jend) ? P::cost(p, i, j + q) : 0.f;
  }
}

template <class P>
__global__ void __launch_bounds__(PINS_TPB, 2)
k_row_lse_mx(PassArgs p, int seg, MergeWS ws, double* F_out, double* out_res) {
  extern __shared__ __align__(16) float2 sB[];
  __shared__ double sh_red[PINS_WARPS];
  __shared__ unsigned long long s_bar[PINS_WARPS][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = p.m, n = p.n;
  const int x = blockIdx.x, y = blockIdx.y, SX = gridDim.x, GY = gridDim.y;
  const int j0 = x * seg, j1 = min(n, j0 + seg);
  const float kh = p.kappa2_dd.hi, kl = p.kappa2_dd.lo;
  // log2(e) B_j = G_j log2(e) / eta as a pair (integer split of the FP64 G_j)
  for (int j = j0 + threadIdx.x; j < j1; j += PINS_TPB) sB[j - j0] = ddv_mul(split_f64(p.G[j], 0), p.l2e_eta);
  __syncthreads();
  // full 1024-column segments of a dense cost: every warp streams its row
  // segments (4 KB each) through two shared-memory buffers with bulk async
  // copies, the next row's copy in flight while the current row is reduced
  const bool full8 = std::is_same<P, PolMixed<COST_DENSE>>::value && (n & 3) == 0 &&
                     seg == 8 * 128 && j1 - j0 == 8 * 128 &&
                     (reinterpret_cast<uintptr_t>(p.cost.C32) & 15u) == 0;
  if (full8) {
    float* wbuf = reinterpret_cast<float*>(sB + seg) + warp * 2 * 1024;
    if (threadIdx.x == 0) {
      for (int w = 0; w < PINS_WARPS; ++w) { mbar_init(&s_bar[w][0], 1); mbar_init(&s_bar[w][1], 1); }
      fence_mbar_init();
      fence_proxy_async();
    }
    __syncthreads();
    const int i_first = y * PINS_WARPS + warp, stride = GY * PINS_WARPS;
    const int T = (i_first < m) ? (m - i_first + stride - 1) / stride : 0;
    if (lane == 0 && T > 0) {
      mbar_expect_tx(&s_bar[warp][0], 4096u);
      bulk_g2s(wbuf, p.cost.C32 + (size_t)i_first * n + j0, 4096u, &s_bar[warp][0]);
    }
    bool ok = true;
    int fail_t = -1;                    // first row whose wait gave up
    for (int t = 0; t < T; ++t) {
      const int i = i_first + t * stride;
      // the buffer of row t - 1 was released by __syncwarp; no copy is issued
      // once a wait of lane 0 has given up
      if (lane == 0 && ok && t + 1 < T) {
        fence_proxy_async();
        mbar_expect_tx(&s_bar[warp][(t + 1) & 1], 4096u);
        bulk_g2s(wbuf + ((t + 1) & 1) * 1024, p.cost.C32 + (size_t)(i + stride) * n + j0, 4096u,
                 &s_bar[warp][(t + 1) & 1]);
      }
      // a wait that gives up (never expected) is recorded; later rows then skip
      // their waits so the pass still ends.  The outcome is made warp-uniform:
      // if any lane gave up, every lane stops waiting and lane 0 issues no
      // further copy, so the drain below covers every lane's failure.
      if (ok) {
        const bool waited = mbar_wait_bounded(&s_bar[warp][t & 1], (unsigned int)((t >> 1) & 1), 1u << 22);
        if (!__all_sync(0xffffffffu, waited)) {
          ok = false;
          fail_t = t;
        }
      }
      const float* rowbuf = wbuf + (t & 1) * 1024;
      float M = -INFINITY, S = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int col = 4 * lane + 128 * k;
        const float4 cv = *reinterpret_cast<const float4*>(rowbuf + col);
        float wh[4], wl[4];
        dd_w(sB[col + 0], cv.x, kh, kl, wh[0], wl[0]);
        dd_w(sB[col + 1], cv.y, kh, kl, wh[1], wl[1]);
        dd_w(sB[col + 2], cv.z, kh, kl, wh[2], wl[2]);
        dd_w(sB[col + 3], cv.w, kh, kl, wh[3], wl[3]);
        lse2_chunk(M, S, wh, wl);
      }
      __syncwarp();
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float Mo = __shfl_xor_sync(0xffffffffu, M, o);
        const float So = __shfl_xor_sync(0xffffffffu, S, o);
        lse2_merge(M, S, Mo, So);
      }
      if (lane == 0) store_f2(ws.rowpart0 + (size_t)x * m + i, M, S);
    }
    if (!ok && p.err) atomicOr(p.err, 16);
    // before the warp leaves its buffers, lane 0 waits (again bounded) for the
    // copies it may still have in flight: the one whose wait gave up and the
    // prefetch issued just before that wait
    if (lane == 0 && !ok) {
      mbar_wait_bounded(&s_bar[warp][fail_t & 1], (unsigned int)((fail_t >> 1) & 1), 1u << 22);
      if (fail_t + 1 < T)
        mbar_wait_bounded(&s_bar[warp][(fail_t + 1) & 1], (unsigned int)(((fail_t + 1) >> 1) & 1),
                          1u << 22);
    }
  }
  for (int i = y * PINS_WARPS + warp; !full8 && i < m; i += GY * PINS_WARPS) {
    float M = -INFINITY, S = 0.f;
    int jb = j0 + 4 * lane;
    // two chunks of 4 per step: both loads issued before either update
    for (; jb + 128 + 3 < j1; jb += 256) {
      float c0[4], c1[4];
      cost4<P>(p, i, jb, j1, c0);
      cost4<P>(p, i, jb + 128, j1, c1);
      float wh[4], wl[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) dd_w(sB[jb + q - j0], c0[q], kh, kl, wh[q], wl[q]);
      lse2_chunk(M, S, wh, wl);
#pragma unroll
      for (int q = 0; q < 4; ++q) dd_w(sB[jb + 128 + q - j0], c1[q], kh, kl, wh[q], wl[q]);
      lse2_chunk(M, S, wh, wl);
    }
    for (; jb < j1; jb += 128) {
      float c[4];
      cost4<P>(p, i, jb, j1, c);
      if (jb + 3 < j1) {
        float wh[4], wl[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) dd_w(sB[jb + q - j0], c[q], kh, kl, wh[q], wl[q]);
        lse2_chunk(M, S, wh, wl);
      } else {
        for (int q = 0; jb + q < j1; ++q) {
          float wh, wl;
          dd_w(sB[jb + q - j0], c[q], kh, kl, wh, wl);
          lse2_one(M, S, wh, wl);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float Mo = __shfl_xor_sync(0xffffffffu, M, o);
      const float So = __shfl_xor_sync(0xffffffffu, S, o);
      lse2_merge(M, S, Mo, So);
    }
    if (lane == 0) store_f2(ws.rowpart0 + (size_t)x * m + i, M, S);
  }
  // merge the segments of this row group (last of its SX CTAs)
  if (arrive_last(ws.cnt_row + y, SX)) {
    const double LN2 = 0.69314718055994530942;
    double res = 0.0;
    const int per = PINS_WARPS * ((m + GY * PINS_WARPS - 1) / (GY * PINS_WARPS));
    for (int k = threadIdx.x; k < per; k += PINS_TPB) {
      const int i = y * PINS_WARPS + (k % PINS_WARPS) + (k / PINS_WARPS) * GY * PINS_WARPS;
      if (i >= m) continue;
      float Mf = -INFINITY, Sf = 0.f;
      for (int xs = 0; xs < SX; ++xs) {
        const float2 o = load_f2_cg(ws.rowpart0 + (size_t)xs * m + i);
        lse2_merge(Mf, Sf, o.x, o.y);
      }
      const double lse2 = (double)Mf + log2((double)Sf);         // base-2 LSE_j of w
      const double A2 = (p.F[i] * p.inv_eta - p.s) * 1.4426950408889634074;
      const double ai = p.a[i];
      if (out_res) res += fabs(exp2(A2 + lse2) - ai);
      F_out[i] = p.eta * (log(ai) + p.s - LN2 * lse2);
    }
    const double br = block_sum(res, sh_red);
    if (threadIdx.x == 0) ws.scal_row[y] = br;
  }
  // the residual (read by the caller only at the end of a block of iterations)
  // is skipped, with its FP64 exp2 per row, when out_res is NULL
  if (out_res && arrive_last(ws.cnt_all, SX * GY)) {
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
  extern __shared__ float2 sA[];                 // log2(e) A_i of the row block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = p.m, n = p.n;
  const int i0 = blockIdx.y * rb, i1 = min(m, i0 + rb);
  const int nct = (n + PINS_TC - 1) / PINS_TC;
  const float kh = p.kappa2_dd.hi, kl = p.kappa2_dd.lo;
  for (int i = i0 + threadIdx.x; i < i1; i += PINS_TPB) sA[i - i0] = a2_of(p, i);
  __syncthreads();
  for (int ct = blockIdx.x; ct < nct; ct += gridDim.x) {
    const int jb = ct * PINS_TC + 4 * lane;
    const int nv = min(4, n - jb);                 // valid columns of this lane (may be <= 0)
    float M[4], S[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) { M[q] = -INFINITY; S[q] = 0.f; }
    if (nv >= 4) {
      int i = i0 + warp;
      // four rows per step: loads first, then a chunk update per column
      for (; i + 3 * PINS_WARPS < i1; i += 4 * PINS_WARPS) {
        float c[4][4];
        float2 A[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          A[t] = sA[i + t * PINS_WARPS - i0];
          cost4<P>(p, i + t * PINS_WARPS, jb, n, c[t]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float wh[4], wl[4];
#pragma unroll
          for (int t = 0; t < 4; ++t) dd_w(A[t], c[t][q], kh, kl, wh[t], wl[t]);
          lse2_chunk(M[q], S[q], wh, wl);
        }
      }
      for (; i < i1; i += PINS_WARPS) {
        float c[4];
        const float2 A = sA[i - i0];
        cost4<P>(p, i, jb, n, c);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float wh, wl;
          dd_w(A, c[q], kh, kl, wh, wl);
          lse2_one(M[q], S[q], wh, wl);
        }
      }
    } else if (nv > 0) {
      for (int i = i0 + warp; i < i1; i += PINS_WARPS) {
        float c[4];
        const float2 A = sA[i - i0];
        cost4<P>(p, i, jb, n, c);
        for (int q = 0; q < nv; ++q) {
          float wh, wl;
          dd_w(A, c[q], kh, kl, wh, wl);
          lse2_one(M[q], S[q], wh, wl);
        }
      }
    }
    // merge the 8 warps per column, in warp order
#pragma unroll
    for (int q = 0; q < 4; ++q) stg[warp][4 * lane + q] = make_float2(M[q], S[q]);
    __syncthreads();
    if (threadIdx.x < PINS_TC) {
      float Mc = -INFINITY, Sc = 0.f;
#pragma unroll
      for (int w = 0; w < PINS_WARPS; ++w) lse2_merge(Mc, Sc, stg[w][threadIdx.x].x, stg[w][threadIdx.x].y);
      const int j = ct * PINS_TC + threadIdx.x;
      if (j < n) store_f2(ws.colpart0 + (size_t)blockIdx.y * n + j, Mc, Sc);
    }
    __syncthreads();
  }
  // merge the row blocks of this CTA's strips (last of the gridDim.y CTAs)
  if (arrive_last(ws.cnt_col + blockIdx.x, gridDim.y)) {
    const double LN2 = 0.69314718055994530942;
    for (int ct = blockIdx.x; ct < nct; ct += gridDim.x) {
      const int j = ct * PINS_TC + threadIdx.x;
      if (threadIdx.x < PINS_TC && j < n) {
        float Mf = -INFINITY, Sf = 0.f;
        for (int yb = 0; yb < (int)gridDim.y; ++yb) {
          const float2 o = load_f2_cg(ws.colpart0 + (size_t)yb * n + j);
          lse2_merge(Mf, Sf, o.x, o.y);
        }
        G_out[j] = p.eta * (log(p.b[j]) - LN2 * ((double)Mf + log2((double)Sf)));
      }
    }
  }
}

}  // namespace pins
