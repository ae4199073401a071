// Shared device-side definitions of the PINS kernels (sm_103a).
//
// Notation (Algorithm 2 with the accumulated potentials of the outer loop):
//   z_ij = log X~_ij = (F_i + G_j - s (C_ij + eta)) / eta = A_i + B_j - kappa C_ij
//   with A_i = F_i / eta - s, B_j = G_j / eta, kappa = s / eta.
// Two arithmetic policies evaluate the m x n passes:
//   PolF64   : IEEE FP64 throughout (FP64 exp).
//   PolMixed : FP32 units only.  The exponent is formed in double-float
//              (hi + lo FP32 pairs), so its error stays ~2^-46 |z| although
//              |A|, |B|, |kappa C| reach 1e5; the Sinkhorn warm-up then takes
//              FP32 ex2, the accurate passes take a double-float exp.
// Keys ranked by Sparsify are F_i + G_j - s (C_ij + eta) in FP64 (same operation
// order as the plain definition, no contraction) or the FP32 value of z.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#define PINS_TPB 256          // threads per block of the m x n pass kernels
#define PINS_WARPS (PINS_TPB / 32)
#define PINS_CPL 4            // columns per lane in a tile
#define PINS_TC (32 * PINS_CPL)   // tile width (columns)
#define PINS_RPT 8            // rows per thread in a tile
#define PINS_TR (PINS_WARPS * PINS_RPT)  // tile height (rows)
#define PINS_GX_MAX 32        // column-strip CTAs (row partial fan-in)
#define PINS_GY_MAX 64        // row-block CTAs (column partial fan-in)
#define PINS_EXP_TABLE 1024   // entries of the 2^(k/1024) table
#define PINS_ROW_GROUPS 256   // arrival counters for row groups (cnt_row)

namespace pins {

// ------------------------------------------------------------------------- //
// double-float (FP32 pair) arithmetic: Knuth TwoSum, FMA-based TwoProduct
// (Ogita, Rump & Oishi 2005), Dekker Fast2Sum.
// ------------------------------------------------------------------------- //
struct dd { float hi, lo; };

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
__device__ __forceinline__ dd dd_from_double(double v) {
  dd r; r.hi = __double2float_rn(v); r.lo = __double2float_rn(v - (double)r.hi); return r;
}
__device__ __forceinline__ double dd_to_double(dd v) { return (double)v.hi + (double)v.lo; }
// a + b for normalised pairs, result normalised
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  float s, e; two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  dd r; fast_two_sum(s, e, r.hi, r.lo); return r;
}
// accumulate a (possibly unnormalised) pair into a running sum
__device__ __forceinline__ void dd_acc(dd& acc, float hi, float lo) {
  float s, e; two_sum(acc.hi, hi, s, e);
  acc.hi = s; acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, lo));
}
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  float p, e; two_prod(a.hi, b.hi, p, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  dd r; fast_two_sum(p, e, r.hi, r.lo); return r;
}

// FP64 -> double-float with integer operations only: hi = the sign, exponent and
// top 23 stored significand bits (truncated), lo = the remaining 29 bits rounded
// to FP32, so hi + lo carries ~48 significand bits.  The binary exponent is
// lowered by `shift` (an exact scaling by 2^-shift).  Zero, FP64 subnormals and
// scaled magnitudes below 2^-126 give 0; above 2^128 give inf; NaN stays NaN.
__device__ __forceinline__ float2 split_f64(double v, int shift) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ffu);
  const unsigned long long mant = b & 0xfffffffffffffull;
  if (e == 0x7ff) return make_float2(__uint_as_float(sign | 0x7f800000u | (mant ? 0x400000u : 0u)), 0.f);
  const int fe = e - 1023 + 127 - shift;
  if (e == 0 || fe <= 0) return make_float2(__uint_as_float(sign), 0.f);
  if (fe >= 255) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.f);
  const float hi = __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)(mant >> 29));
  const unsigned rest = (unsigned)(mant & 0x1fffffffu);
  // rest * 2^-52 is exact and normal; times 2^(fe - 127) may round if subnormal
  float lo = __fmul_rn(__fmul_rn(__uint2float_rn(rest), 0x1p-52f), __uint_as_float((unsigned)fe << 23));
  if (sign) lo = -lo;
  return make_float2(hi, lo);
}

__device__ __forceinline__ float2 ddv_mul(float2 a, float2 b) {
  float p, e; two_prod(a.x, b.x, p, e);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  float h, l; fast_two_sum(p, e, h, l);
  return make_float2(h, l);
}
// f * v (f FP32, v double-float), normalised
__device__ __forceinline__ float2 ddv_scale(float f, float2 v) {
  float p, e; two_prod(f, v.x, p, e);
  e = __fmaf_rn(f, v.y, e);
  float h, l; fast_two_sum(p, e, h, l);
  return make_float2(h, l);
}
__device__ __forceinline__ float2 ddv_neg(float2 a) { return make_float2(-a.x, -a.y); }
// a / b for double-float a, b: an FP32 quotient of the leading parts corrected
// by the remainder a - q b (formed exactly by TwoProduct), normalised.  The
// correction absorbs the error of the fast reciprocal quotient.
__device__ __forceinline__ float2 ddv_div(float2 a, float2 b) {
  const float ib = __frcp_rn(b.x);
  const float q1 = __fmul_rn(a.x, ib);
  float p, e; two_prod(q1, b.x, p, e);
  e = __fmaf_rn(q1, b.y, e);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.x, p), e), a.y);
  const float q2 = __fmul_rn(r, ib);
  float h, l; fast_two_sum(q1, q2, h, l);
  return make_float2(h, l);
}
// y + f * v  (f FP32, v and y double-float), normalised
__device__ __forceinline__ float2 ddv_axpy(float f, float2 v, float2 y) {
  float p, e; two_prod(f, v.x, p, e);
  e = __fmaf_rn(f, v.y, e);
  float s, t; two_sum(y.x, p, s, t);
  t = __fadd_rn(t, __fadd_rn(y.y, e));
  float h, l; fast_two_sum(s, t, h, l);
  return make_float2(h, l);
}
// f v + y with f, v, y double-float (the product's f.y v.y term dropped)
__device__ __forceinline__ float2 ddv_axpy2(float2 f, float2 v, float2 y) {
  float p, e; two_prod(f.x, v.x, p, e);
  e = __fmaf_rn(f.x, v.y, __fmaf_rn(f.y, v.x, e));
  float s, t; two_sum(y.x, p, s, t);
  t = __fadd_rn(t, __fadd_rn(y.y, e));
  float h, l; fast_two_sum(s, t, h, l);
  return make_float2(h, l);
}
// acc += v * u (v double-float, u FP32), unnormalised accumulation
__device__ __forceinline__ void ddv_acc_mul(float2& acc, float2 v, float u) {
  float p, e; two_prod(v.x, u, p, e);
  e = __fmaf_rn(v.y, u, e);
  float s, t; two_sum(acc.x, p, s, t);
  acc.x = s; acc.y = __fadd_rn(acc.y, __fadd_rn(t, e));
}
__device__ __forceinline__ float2 ddv_add(float2 a, float2 b) {
  float s, t; two_sum(a.x, b.x, s, t);
  t = __fadd_rn(t, __fadd_rn(a.y, b.y));
  float h, l; fast_two_sum(s, t, h, l);
  return make_float2(h, l);
}

// exp of a double-float argument, double-float result with relative error
// about 2^-45 (tested against FP64 exp).  Table-driven method of Tang (ACM TOMS
// 15(2), 1989): z log2(e) = k/1024 + r, exp(z) = 2^(k >> 10) T[k & 1023] e^(r ln 2),
// T[q] = 2^(q/1024) as a double-float pair, e^x - 1 by its Taylor series
// (|x| <= ln2/2048).  Arguments below -87 give 0 (FP32 range), above 88.7 inf.
struct ExpTable { const float2* t; };

__device__ __forceinline__ dd dd_exp(float zh, float zl, const float2* __restrict__ T) {
  const float L1 = 1.44269502162933349609375f;         // log2(e) hi
  const float L2 = 1.925963033500011079e-08f;          // log2(e) - L1
  const float N1 = 0.693145751953125f;                 // ln 2 hi (exact in few bits)
  const float N2 = 1.428606765330187045e-06f;          // ln 2 - N1
  dd out;
  if (!(zh > -87.0f)) { out.hi = 0.f; out.lo = 0.f; return out; }  // also NaN-safe
  if (zh > 88.7f) { out.hi = __int_as_float(0x7f800000); out.lo = 0.f; return out; }
  float p, pe; two_prod(zh, L1, p, pe);
  pe = __fmaf_rn(zh, L2, pe);
  pe = __fmaf_rn(zl, L1, pe);
  float kf = rintf(p * 1024.0f);
  float rh = __fsub_rn(p, kf * (1.0f / 1024.0f));      // exact (Sterbenz)
  // x = (rh + pe) ln 2 as a pair
  float xh, xe; two_prod(rh, N1, xh, xe);
  xe = __fmaf_rn(rh, N2, xe);
  xe = __fmaf_rn(pe, N1, xe);
  float x = xh + xe;
  // q = x^2/2 + x^3/6 + x^4/24
  float q = x * x * __fmaf_rn(x, __fmaf_rn(x, 1.0f / 24.0f, 1.0f / 6.0f), 0.5f);
  int k = (int)kf;
  int qi = k & (PINS_EXP_TABLE - 1);
  int e2 = k >> 10;   // arithmetic shift = floor(k / 1024)
  float2 t = T[qi];
  // T (1 + xh + xe + q) = T.x + [T.x xh] + T.x (xe + q) + T.y (1 + x)
  float ph, pl; two_prod(t.x, xh, ph, pl);
  pl = __fmaf_rn(t.x, xe + q, pl);
  pl = __fmaf_rn(t.y, 1.0f + x, pl);
  float sh, sl; fast_two_sum(t.x, ph, sh, sl);
  sl = __fadd_rn(sl, pl);
  // scale by 2^e2 (split in two factors to stay within the normal range)
  int e2a = e2 >> 1, e2b = e2 - e2a;
  float fa = __int_as_float((e2a + 127) << 23);
  float fb = __int_as_float((e2b + 127) << 23);
  out.hi = sh * fa * fb;
  out.lo = sl * fa * fb;
  return out;
}

// expm1(y) - y in FP32 with small relative error for every y: Taylor series
// y^2 (1/2! + y/3! + ... + y^8/10!) for |y| < 1/2 (remainder below 1e-10
// relative), expf(y) - 1 - y beyond (relative error below ~1e-6).
__device__ __forceinline__ float expm1_minus_x(float y) {
  if (fabsf(y) < 0.5f) {
    float p = 1.0f / 3628800.0f;
    p = __fmaf_rn(p, y, 1.0f / 362880.0f);
    p = __fmaf_rn(p, y, 1.0f / 40320.0f);
    p = __fmaf_rn(p, y, 1.0f / 5040.0f);
    p = __fmaf_rn(p, y, 1.0f / 720.0f);
    p = __fmaf_rn(p, y, 1.0f / 120.0f);
    p = __fmaf_rn(p, y, 1.0f / 24.0f);
    p = __fmaf_rn(p, y, 1.0f / 6.0f);
    p = __fmaf_rn(p, y, 0.5f);
    return __fmul_rn(__fmul_rn(y, y), p);
  }
  return __fsub_rn(__fsub_rn(expf(y), 1.0f), y);
}

// Line-search objective term X~ (expm1(t) - t) >= 0 of one entry (mixed
// policy), from z0 = log X~ (FP32), t and e1 = X~ e^t (the trial entry, already
// formed in double-float).  For |t| < 1/2 the series form is free of
// cancellation; otherwise the term is e1 - X~ (1 + t), which loses at most a
// few bits there and stays finite when X~ underflows FP32 (z0 < -87) while e^t
// alone would overflow.
__device__ __forceinline__ float trial_term(float z0, float t, float e1) {
  const float x0 = (z0 > -87.0f) ? exp2f(__fmul_rn(z0, 1.4426950408889634f)) : 0.0f;
  if (fabsf(t) < 0.5f) return __fmul_rn(x0, expm1_minus_x(t));
  return fmaxf(0.0f, __fsub_rn(e1, __fmul_rn(x0, __fadd_rn(1.0f, t))));
}

// expm1 of a double-float argument with relative accuracy ~2^-44 for small |t|.
__device__ __forceinline__ dd dd_expm1(float th, float tl, const float2* __restrict__ T) {
  dd r;
  if (fabsf(th) < (1.0f / 1024.0f)) {
    // t + t^2/2 + t^3/6 + t^4/24 + t^5/120 with t^2 kept as a pair
    float p, pe; two_prod(th, th, p, pe);
    float t3 = p * th;
    float tail = __fmaf_rn(t3, __fmaf_rn(th, __fmaf_rn(th, 1.0f / 120.0f, 1.0f / 24.0f), 1.0f / 6.0f),
                           0.5f * pe + th * tl);
    // th + 0.5 p + (tl + tail)
    float s, e; fast_two_sum(th, 0.5f * p, s, e);
    r.hi = s; r.lo = __fadd_rn(e, __fadd_rn(tl, tail));
    float h, l; fast_two_sum(r.hi, r.lo, h, l); r.hi = h; r.lo = l;
    return r;
  }
  dd e = dd_exp(th, tl, T);
  if (isinf(e.hi)) return e;
  float s, err; two_sum(e.hi, -1.0f, s, err);
  r.hi = s; r.lo = __fadd_rn(err, e.lo);
  float h, l; fast_two_sum(r.hi, r.lo, h, l); r.hi = h; r.lo = l;
  return r;
}

// ------------------------------------------------------------------------- //
// Bulk asynchronous copies (TMA engine) from global to shared memory, completed
// on a shared-memory mbarrier.  Addresses 16-byte aligned, sizes multiples of 16.
// ------------------------------------------------------------------------- //
__device__ __forceinline__ unsigned int smem_u32(const void* p) {
  return (unsigned int)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// orders shared-memory accesses of the threads (generic proxy) before later
// accesses of the copy engine (async proxy)
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// makes barrier initialisations visible before their first use
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned int bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned int bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned int parity) {
  unsigned int ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false after `limit` polls (the caller records the failure)
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned int parity,
                                                  unsigned int limit) {
  for (unsigned int k = 0; k < limit; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// ------------------------------------------------------------------------- //
// warp / block reductions
// ------------------------------------------------------------------------- //
// double-float butterfly sum (every lane gets the total; fixed order)
__device__ __forceinline__ dd warp_dd_sum(dd v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dd w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = dd_add(v, w);
  }
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_maxf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_maxd(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_mind(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// float pairs stored raw in an 8-byte partial slot (mixed policy: no FP64 ops)
__device__ __forceinline__ void store_f2(double* slot, float x, float y) {
  *reinterpret_cast<float2*>(slot) = make_float2(x, y);
}
__device__ __forceinline__ float2 load_f2(const double* slot) {
  return *reinterpret_cast<const float2*>(slot);
}
__device__ __forceinline__ float2 load_f2_cg(const double* slot) {
  double v = __ldcg(slot);
  return *reinterpret_cast<float2*>(&v);
}
// FP32 LSE pair merge
__device__ __forceinline__ void lse_merge_f(float& m1, float& s1, float m2, float s2) {
  if (m2 == -INFINITY) return;
  if (m1 == -INFINITY) { m1 = m2; s1 = s2; return; }
  if (m2 > m1) { s1 = s1 * exp2f((m1 - m2) * 1.4426950408889634f) + s2; m1 = m2; }
  else { s1 = s1 + s2 * exp2f((m2 - m1) * 1.4426950408889634f); }
}
// LSE pair merge: (m1, s1) <- (m1, s1) (+) (m2, s2); m = -inf means empty
__device__ __forceinline__ void lse_merge(double& m1, double& s1, double m2, double s2) {
  if (m2 == -INFINITY) return;
  if (m1 == -INFINITY) { m1 = m2; s1 = s2; return; }
  if (m2 > m1) { s1 = s1 * exp(m1 - m2) + s2; m1 = m2; }
  else { s1 = s1 + s2 * exp(m2 - m1); }
}

// ------------------------------------------------------------------------- //
// Cost sources.  c64(i,j): the cost C_ij in FP64, evaluated exactly as the
// plain definition (dense read, or scale * sum of squared differences, or
// scale * integer squared grid distance), with no contraction.
// c32(i,j): an FP32 "raw" cost c' with C_ij = cscale * c'.
// ------------------------------------------------------------------------- //
enum CostKind { COST_DENSE = 0, COST_POINTS = 1, COST_GRID = 2 };

struct CostArgs {
  int kind;
  int m, n, d;
  const double* C64;   // dense FP64
  const float* C32;    // dense FP32
  const double* x;     // points FP64 (m*d)
  const double* y;     // points FP64 (n*d)
  const float* xf;     // points FP32
  const float* yf;
  double scale;        // points / grid
  int s2;              // grid width
};

template <int KIND> struct Cost64;
template <> struct Cost64<COST_DENSE> {
  __device__ __forceinline__ static double c(const CostArgs& a, int i, int j) {
    return __ldg(a.C64 + (size_t)i * a.n + j);
  }
};
template <> struct Cost64<COST_POINTS> {
  __device__ __forceinline__ static double c(const CostArgs& a, int i, int j) {
    const double* xi = a.x + (size_t)i * a.d;
    const double* yj = a.y + (size_t)j * a.d;
    double d0 = __dsub_rn(__ldg(xi), __ldg(yj));
    double acc = __dmul_rn(d0, d0);
    for (int q = 1; q < a.d; ++q) {
      double dq = __dsub_rn(__ldg(xi + q), __ldg(yj + q));
      acc = __dadd_rn(acc, __dmul_rn(dq, dq));
    }
    return __dmul_rn(a.scale, acc);
  }
};
template <> struct Cost64<COST_GRID> {
  __device__ __forceinline__ static double c(const CostArgs& a, int i, int j) {
    int d1 = i / a.s2 - j / a.s2, d2 = i % a.s2 - j % a.s2;
    return __dmul_rn(a.scale, (double)(d1 * d1 + d2 * d2));
  }
};

template <int KIND> struct Cost32;
template <> struct Cost32<COST_DENSE> {
  __device__ __forceinline__ static float c(const CostArgs& a, int i, int j) {
    return __ldg(a.C32 + (size_t)i * a.n + j);
  }
};
template <> struct Cost32<COST_POINTS> {
  __device__ __forceinline__ static float c(const CostArgs& a, int i, int j) {
    const float* xi = a.xf + (size_t)i * a.d;
    const float* yj = a.yf + (size_t)j * a.d;
    float acc = 0.f;
    for (int q = 0; q < a.d; ++q) {
      float dq = __ldg(xi + q) - __ldg(yj + q);
      acc = __fmaf_rn(dq, dq, acc);
    }
    return acc;
  }
};
template <> struct Cost32<COST_GRID> {
  __device__ __forceinline__ static float c(const CostArgs& a, int i, int j) {
    int d1 = i / a.s2 - j / a.s2, d2 = i % a.s2 - j % a.s2;
    return (float)(d1 * d1 + d2 * d2);
  }
};

// ------------------------------------------------------------------------- //
// Per-pass scalar parameters shared by every m x n kernel.
// ------------------------------------------------------------------------- //
struct PassArgs {
  CostArgs cost;
  int m, n;
  double eta, inv_eta, s;
  double kappa;          // s / eta  (FP64 path)
  dd kappa_dd;           // kappa * cost scale of the FP32 raw cost (mixed path)
  double cscale;         // C_ij = cscale * c32(i,j) on the mixed path
  const double* F; const double* G;       // potentials
  const double* A64; const double* B64;   // FP64: A = F/eta - s, B = G/eta
  const float2* Add; const float2* Bdd;   // mixed: same as double-float pairs
  float2 l2e_eta;                         // mixed Sinkhorn: log2(e) / eta as a pair
  float2 s_l2e;                           // s log2(e) as a pair
  dd kappa2_dd;                           // log2(e) kappa_dd
  const double* a; const double* b;
  const double* la; const double* lb;     // log a, log b (mixed grid half-steps; else NULL)
  const float2* exp_table;                // 2^(q/1024) pairs (mixed)
  int* err;                               // bit 4: a bulk-copy wait gave up (may be NULL)
};

// Geometry of the tiled passes.
struct TileGeom {
  int nct, nrt;   // column tiles, row tiles
  int gx, gy;     // grid dims (strips, row blocks)
};

__host__ __device__ inline TileGeom make_geom(int m, int n) {
  TileGeom g;
  g.nct = (n + PINS_TC - 1) / PINS_TC;
  g.nrt = (m + PINS_TR - 1) / PINS_TR;
  g.gx = g.nct < PINS_GX_MAX ? g.nct : PINS_GX_MAX;
  g.gy = g.nrt < PINS_GY_MAX ? g.nrt : PINS_GY_MAX;
  return g;
}

// Cross-CTA merge bookkeeping (deterministic "last block" pattern).
struct MergeWS {
  unsigned int* cnt_row;   // PINS_ROW_GROUPS counters (arrivals of the strips of a row group)
  unsigned int* cnt_col;   // gx counters (arrivals of gy row blocks)
  unsigned int* cnt_all;   // 1 counter (arrivals of gx*gy CTAs)
  double* rowpart0;        // gx * m
  double* rowpart1;        // gx * m
  double* rowpart2;        // gx * m
  double* rowpart3;        // gx * m
  double* rowpart4;        // gx * m
  double* rowpart5;        // gx * m (certificate only)
  double* colpart0;        // gy * n
  double* colpart1;        // gy * n
  double* colpart2;        // gy * n (certificate only)
  double* scal_row;        // gy * 8 per-row-block scalar partials
  double* scal_col;        // gx * 8 per-strip scalar partials
};

}  // namespace pins
