// m x n pass kernels of PINS, templated on the arithmetic policy (FP64 or
// mixed) and the cost source.  Every pass tiles the matrix into 64 x 128 tiles;
// a CTA owns one column strip x and one row block y and loops over the tiles
// congruent to (x, y).  Row results are merged across strips and column results
// across row blocks by the last CTA to arrive.  The merges stage the partials
// in shared memory with independent coalesced loads and reduce them in a fixed
// order, so every result is bit-reproducible regardless of scheduling or of
// other work on the device.
//
// GB300 note: a warp-wide FP64 instruction occupies the FP64 pipe for ~64
// cycles, so the mixed policy keeps every per-entry and per-row step on the
// FP32 units (double-float pairs stored raw in the 8-byte partial slots) and
// converts to FP64 once per row or column at the end of a merge.
#pragma once
#include <type_traits>
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

// fixed-tree block reductions (result valid in thread 0)
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
  return r;
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

// Stages `cnt` slices of `width` consecutive 8-byte partials (slice s starts at
// base + s * stride) into smem[s * width + c]; c >= valid is zero-filled.  All
// loads are independent and coalesced (bypassing L1: written by other CTAs).
#define PINS_STAGE (PINS_GX_MAX * PINS_TR)   // 2048 slots = 16 KiB
__device__ __forceinline__ void stage8(const double* base, size_t stride, int cnt, int width,
                                       int valid, double* smem) {
  for (int k = threadIdx.x; k < cnt * width; k += PINS_TPB) {
    const int s = k / width, c = k - s * width;
    smem[k] = (c < valid) ? __ldcg(base + (size_t)s * stride + c) : 0.0;
  }
}
__device__ __forceinline__ float2 as_f2(double v) { return *reinterpret_cast<float2*>(&v); }

}  // namespace pins

#include "pins_pass_lse.cuh"
#include "pins_pass_lse_mx.cuh"
#include "pins_pass_grid_lse.cuh"
#include "pins_pass_marg.cuh"
#include "pins_pass_marg_mx.cuh"
#include "pins_pass_cert.cuh"
#include "pins_tree.cuh"
