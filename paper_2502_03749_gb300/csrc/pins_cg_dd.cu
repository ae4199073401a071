// Truncated Jacobi-preconditioned CG of the Newton step (Algorithm 2) for the
// mixed-precision path: one thread-block cluster, every vector resident in
// shared memory, all vector arithmetic in double-float (FP32 pairs).
//
// Why double-float: this GPU issues FP64 at ~1/70 of its FP32 rate, and a CG
// iteration on a few thousand unknowns is a chain of short dependent steps, so
// FP64 latency sets its length.  Every vector, the matrix-vector product
// (diagonal and S entries scaled by 1/eta) and the three inner products per
// iteration (r.u, w.u, r.r) keep ~48 significand bits; the step lengths alpha,
// beta are formed and applied in double-float (the same value in every
// recurrence, so the recurrences stay consistent).  FP32
// inner products, measured on the Newton systems of 64 x 64 grid problems,
// doubled the iteration count against FP64 CG and let the recurrence residual
// drift from the true one by two orders of magnitude.  The preconditioner is
// D^-1 with D^-1 rounded to FP32 (a fixed diagonal).  rhs is scaled by a power
// of two (exact) so that its largest entry is in [1, 2); x is scaled back at
// the end.
//
// Ordering: the single-reduction PCG of Chronopoulos & Gear (J. Comput. Appl.
// Math. 25, 1989), as in the FP64 cluster CG:
//   u = D^-1 r exchanged                                  [arrival, or barrier]
//   w = M u;  (r.u, w.u, r.r) partials published          [cluster barrier]
//   gamma, delta, rr (every CTA, same order);  stop if rr <= rtol^2 rr_0
//   beta = gamma/gamma', alpha = gamma/(delta - beta gamma/alpha')
//   p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s
// In exact arithmetic these are the iterates, and the iteration count, of the
// textbook Jacobi PCG with the same stopping rule.  The pipelined ordering of
// Ghysels & Vanroose (Parallel Computing 40, 2014) saves the second barrier by
// carrying M u, M D^-1 w and two more vectors as recurrences; on the Newton
// systems of grid problems (Jacobi-preconditioned condition numbers that take
// textbook PCG thousands of iterations) those recurrences drift: in FP64 the
// pipelined iteration stalls where the textbook one converges, and here it
// needed 2.6x the textbook iterations with restarts.  The single-reduction
// form follows the textbook count within a few per cent at this precision.
// Each CTA keeps a replica of u over the range of targets its entries read.
// When every CTA has room for its replica, each CTA pushes its new u slice into
// the replicas with shared-to-shared bulk copies that complete on the
// consumer's mbarrier, so the consumer waits for its data alone, not for a
// cluster barrier; otherwise u goes through L2 (one buffer: its reads and
// writes are separated by a barrier each way) and is fetched into the replica
// or gathered from L2.  The block partials go through distributed shared
// memory (two alternating slot sets).  A system small enough for one CTA runs
// in a cluster of one, which reads u from its own shared memory.
// Every CTA sums the block partials in the same order and takes the same
// decisions, so results are reproducible run to run.
#include <cooperative_groups.h>
#include "pins_kernels.h"
#include "pins_common.cuh"

namespace cg = cooperative_groups;

namespace pins {

#define PINS_DDCG_MAX 16
#define PINS_DDCG_TPB 256
#define PINS_DDCG_SMEM (220 * 1024)
// cluster size: one CTA up to PINS_DDCG_LOCAL_MAX unknowns (no exchange through
// L2, no cluster barrier), else at most PINS_DDCG_SLICE unknowns per CTA where
// the cluster size allows.  Measured on GB300: a 1-CTA CG on 512 unknowns takes
// 3.7 us per iteration against 3.9-5.7 us for 2-16 CTAs; on 2048 unknowns 8 CTAs
// (4.1 us) beat 4 (4.5 us) and 16 (4.5 us); on 8192, 16 CTAs (5.9 us) beat 8 (7.1 us).
#define PINS_DDCG_LOCAL_MAX 512
#define PINS_DDCG_SLICE 256
// shared bytes per unknown: x, r, u, w, s, p, diag, od (8 x 8) + D^-1 (4) + row begin (4)
#define PINS_DDCG_PER_UNKNOWN 72
// passes of the CG: the first, and restarts from x when the true residual at
// the end of a pass is above twice the tolerance
#define PINS_DDCG_PASSES 4
// weight of an unknown against an entry in the work balance of the slices
#ifndef PINS_DDCG_UW
#define PINS_DDCG_UW 2
#endif

struct CGddArgs {
  int m, n;
  double inv_eta;
  const double* r; const double* c;
  const int* indptr; const int* indices; const double* data;
  const int* colptr; const int* rowidx; const double* cdata;
  const double* rhs; double* x;
  const double* ab;                // (a; b): with rhs == NULL, rhs = (a - r; b - c)
  double* dots;                    // if not NULL: <rhs, x> and <ab, x> (FP64, fixed order)
  int* ent_tgt; float2* ent_val;   // scratch: one slot per entry of the CSR + CSC entry space
  int* ent_row;
  float* ug;                       // exchange buffers: u, then x (2 N double-float pairs)
  size_t smem_bytes;               // dynamic shared memory of the launch
  double rtol2; int max_iter; double* info;
  int* flag;                       // bit 0: an entry's target fell outside the cluster's slices;
                                   // bit 7: a bulk-copy wait gave up
};

// longest slice a CTA of a cluster of cs may own: twice the uniform share when
// the shared memory holds it (room for balancing by work), else the share
// (even in a cluster: slice bounds are even, so that slices move in 16-byte
// double-float pairs)
__host__ __device__ inline int ddcg_slice_cap(int N, int cs) {
  const int Lu = (N + cs - 1) / cs;
  if (cs == 1) return Lu;
  const int L2 = 2 * Lu;
  return ((size_t)PINS_DDCG_PER_UNKNOWN * ((L2 + 3) & ~3) + 16 <= PINS_DDCG_SMEM) ? L2
                                                                                  : (Lu + 1) & ~1;
}

// cluster address of a shared-memory location of CTA `rank`
__device__ __forceinline__ unsigned int ddcg_mapa(const void* p, unsigned int rank) {
  unsigned int r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}

// LOCAL: a cluster of one CTA holds every unknown, so the SpMV reads m from its
// own shared memory and nothing goes through the exchange buffer.
template <bool LOCAL>
__global__ void __launch_bounds__(PINS_DDCG_TPB, 1) k_pcg_dd(CGddArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char ddcg_smem[];
  __shared__ float2 slot[2][3][PINS_DDCG_MAX];    // double-buffered block partials
  __shared__ unsigned int eslot[1];
  __shared__ double dred[2][PINS_DDCG_TPB / 32];
  __shared__ double dslot[2][PINS_DDCG_MAX];
  __shared__ float2 red[3][PINS_DDCG_TPB / 32];
  __shared__ unsigned int ered[PINS_DDCG_TPB / 32];
  __shared__ int hrow[PINS_DDCG_TPB];
  __shared__ float2 hval[PINS_DDCG_TPB];
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = a.m, N = a.m + a.n;
  const int Kc = __ldg(a.indptr + m);
  auto beg = [&](int t) -> int {
    return (t < m) ? __ldg(a.indptr + t) : Kc + __ldg(a.colptr + t - m);
  };
  // Slices balanced by work: unknowns [b_k, b_{k+1}) go to CTA k, with b_k the
  // first even unknown at or below the one whose cumulative cost (entries
  // before it + PINS_DDCG_UW per unknown before it) reaches k/CS of the total,
  // each slice at most Lcap long.  Every CTA computes the same boundaries.
  __shared__ int sbound[PINS_DDCG_MAX + 1];
  const int Lcap = ddcg_slice_cap(N, CS);
  if (warp == 0) {
    const long long total = (long long)beg(N) + (long long)PINS_DDCG_UW * N;
    int bk = 0;
    if (lane > 0 && lane < CS) {
      const long long target = (total * lane + CS - 1) / CS;
      int lo_s = 0, hi_s = N;
      while (lo_s < hi_s) {
        const int mid = (lo_s + hi_s) >> 1;
        if ((long long)beg(mid) + (long long)PINS_DDCG_UW * mid >= target) hi_s = mid; else lo_s = mid + 1;
      }
      bk = lo_s & ~1;
    }
    if (lane < CS) sbound[lane] = bk;
    __syncwarp();
    if (lane == 0) {
      sbound[0] = 0;
      for (int k = 1; k < CS; ++k) {
        const int lower = (max(sbound[k - 1], N - (CS - k) * Lcap) + 1) & ~1;
        const int upper = sbound[k - 1] + Lcap;
        sbound[k] = min(max(sbound[k], lower), upper);
      }
      sbound[CS] = N;
    }
  }
  __syncthreads();
  const int lo = sbound[rank];
  const int nl = sbound[rank + 1] - lo;
  // shared memory: the own slice (8 double-float arrays and 1 FP32 array of L4,
  // L4 + 4 row offsets), then, when the dynamic allocation has room, this CTA's
  // packed entries (target, value / eta, local row)
  const int L4 = (Lcap + 3) & ~3;
  float2* xv = reinterpret_cast<float2*>(ddcg_smem);
  float2* rv = xv + L4;
  float2* uv = rv + L4;       // D^-1 r (published in the exchange buffer)
  float2* wv = uv + L4;       // M u
  float2* sv = wv + L4;       // M p (recurrence)
  float2* pv = sv + L4;
  float2* dg = pv + L4;       // diag / eta
  float2* od = dg + L4;       // off-diagonal part of M u (zeroed after use)
  float* dinv = reinterpret_cast<float*>(od + L4);
  int* rb = reinterpret_cast<int*>(dinv + L4);   // nl + 1 entry offsets (relative to E0)
  const size_t base_bytes = sizeof(float) * (size_t)(PINS_DDCG_PER_UNKNOWN / 4) * L4 + 16;
  float2* ug0 = reinterpret_cast<float2*>(a.ug);  // u of every unknown
  float2* ug1 = ug0 + N;                          // x of every unknown (true residual)

  const float2 ie = split_f64(a.inv_eta, 0);
  // the right-hand side: given, or the gradient (a - r; b - c) of the Newton step
  auto rhs_of = [&](int t) -> double {
    if (a.rhs) return a.rhs[t];
    return a.ab[t] - ((t < m) ? __ldg(a.r + t) : __ldg(a.c + t - m));
  };

  // ---- scale: largest binary exponent of rhs over the cluster ----
  unsigned int emax = 0u;
  for (int k = tid; k < nl; k += PINS_DDCG_TPB) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(rhs_of(lo + k));
    emax = max(emax, (unsigned)((b >> 52) & 0x7ffu));
  }
  emax = __reduce_max_sync(0xffffffffu, emax);
  if (lane == 0) ered[warp] = emax;
  __syncthreads();
  if (warp == 0) {
    unsigned int v = lane < PINS_DDCG_TPB / 32 ? ered[lane] : 0u;
    v = __reduce_max_sync(0xffffffffu, v);
    if (lane == 0) eslot[0] = v;                    // read by the other CTAs after the barrier
  }
  // ---- own unknowns: diagonal, preconditioner, residual, row offsets ----
  const int E0 = beg(min(lo, N));
  const int E1 = beg(min(lo + nl, N));
  // ---- entries of the own unknowns: packed (target, value / eta, local row),
  // in shared memory when they fit, else in the global scratch.  Thread t's
  // SpMV share is the local entries [t ne / TPB, (t + 1) ne / TPB); its j-th
  // entry is stored at slot j TPB + t, so one step of a warp reads contiguous
  // words (conflict-free in shared memory, coalesced in global memory).
  const int ne = E1 - E0;
  const int c0 = (int)(((long long)tid * ne) / PINS_DDCG_TPB);
  const int c1 = (int)(((long long)(tid + 1) * ne) / PINS_DDCG_TPB);
  const size_t ent_slots = (size_t)((ne + PINS_DDCG_TPB - 1) / PINS_DDCG_TPB) * PINS_DDCG_TPB;
  auto slot_of = [&](int le) -> int {
    const int t = (int)((((long long)le + 1) * PINS_DDCG_TPB - 1) / ne);
    const int ct = (int)(((long long)t * ne) / PINS_DDCG_TPB);
    return (le - ct) * PINS_DDCG_TPB + t;
  };
  const size_t used = base_bytes;
  const size_t ent_bytes_s = (2 * sizeof(int) + sizeof(float2)) * ent_slots;
  const bool ent_local = used + ent_bytes_s <= a.smem_bytes;
  float2* ev_s = reinterpret_cast<float2*>(ddcg_smem + used);
  int* et_s = reinterpret_cast<int*>(ev_s + ent_slots);
  int* er_s = et_s + ent_slots;
  const size_t gofs = (size_t)E0 + (size_t)rank * PINS_DDCG_TPB;   // padded global region
  int* etg = ent_local ? et_s : a.ent_tgt + gofs;   // target - f0
  float2* eva = ent_local ? ev_s : a.ent_val + gofs;
  int* erow = ent_local ? er_s : a.ent_row + gofs;  // local unknown of each entry
  // the targets this CTA reads lie in [f0, f1) (even bounds: 16-byte aligned
  // copies); a cluster of one reads its own slice and keeps absolute targets
  __shared__ unsigned int tmin_s[PINS_DDCG_TPB / 32], tmax_s[PINS_DDCG_TPB / 32];
  int f0 = 0, f1 = N;
  if (!LOCAL) {
    unsigned int tmin = 0xffffffffu, tmax = 0u;
    for (int e = E0 + tid; e < E1; e += PINS_DDCG_TPB) {
      const int g = (e < Kc) ? m + __ldg(a.indices + e) : __ldg(a.rowidx + e - Kc);
      if (g >= 0 && g < N) { tmin = min(tmin, (unsigned)g); tmax = max(tmax, (unsigned)g); }
    }
    tmin = __reduce_min_sync(0xffffffffu, tmin);
    tmax = __reduce_max_sync(0xffffffffu, tmax);
    if (lane == 0) { tmin_s[warp] = tmin; tmax_s[warp] = tmax; }
    __syncthreads();
    tmin = 0xffffffffu; tmax = 0u;
    for (int w = 0; w < PINS_DDCG_TPB / 32; ++w) { tmin = min(tmin, tmin_s[w]); tmax = max(tmax, tmax_s[w]); }
    if (tmin > tmax) { tmin = 0u; tmax = 0u; }     // no valid entry
    f0 = (int)tmin & ~1;
    f1 = ((int)tmax + 2) & ~1;                      // <= N + 1: inside the two exchange buffers
  }
  // a replica of the exchanged u[f0, f1) in shared memory, filled by bulk copies
  // after each exchange, when the allocation has room after the slice and entries
  const size_t rep_off = (used + (ent_local ? ent_bytes_s : 0) + 15) & ~(size_t)15;
  const unsigned int rep_bytes = (unsigned int)((size_t)(f1 - f0) * sizeof(float2));
  bool rep = !LOCAL && rep_off + rep_bytes <= a.smem_bytes &&
             (reinterpret_cast<uintptr_t>(a.ug) & 15) == 0;
  float2* ur = reinterpret_cast<float2*>(ddcg_smem + rep_off);
  __shared__ __align__(8) unsigned long long rbar;
  unsigned int rpar = 0;
  if (rep && tid == 0) { mbar_init(&rbar, 1); fence_mbar_init(); }
  // replica geometry of this CTA, read by the others after the first barrier
  __shared__ int rinfo[4];                          // f0, f1, replica offset, has replica
  __shared__ int cf0[PINS_DDCG_MAX], cf1[PINS_DDCG_MAX], croff[PINS_DDCG_MAX];
  __shared__ int push_s;
  if (tid == 0) { rinfo[0] = f0; rinfo[1] = f1; rinfo[2] = (int)rep_off; rinfo[3] = rep ? 1 : 0; }
  for (int k = tid; k < nl; k += PINS_DDCG_TPB) {
    const int t = lo + k;
    const double d = (t < m) ? __ldg(a.r + t) : __ldg(a.c + t - m);
    const float2 dd_ = ddv_mul(split_f64(d, 0), ie);
    dg[k] = dd_;
    dinv[k] = __frcp_rn(dd_.x);
    xv[k] = make_float2(0.f, 0.f);
    sv[k] = make_float2(0.f, 0.f);
    pv[k] = make_float2(0.f, 0.f);
    od[k] = make_float2(0.f, 0.f);
    const int b0 = beg(t) - E0, b1 = beg(t + 1) - E0;
    rb[k] = b0;
    for (int e = b0; e < b1; ++e) erow[slot_of(e)] = k;
  }
  if (tid == 0) rb[nl] = E1 - E0;
  for (int e = E0 + tid; e < E1; e += PINS_DDCG_TPB) {
    int g; double v;
    if (e < Kc) { v = __ldg(a.data + e); g = m + __ldg(a.indices + e); }
    else { v = __ldg(a.cdata + e - Kc); g = __ldg(a.rowidx + e - Kc); }
    float2 val = ddv_mul(split_f64(v, 0), ie);
    if (g < 0 || g >= N) {
      atomicOr(a.flag, 1);
      g = f0; val = make_float2(0.f, 0.f);
    }
    const int sl = slot_of(e - E0);
    etg[sl] = g - f0;
    eva[sl] = val;
  }
  // first cluster barrier: every CTA has started (no distributed shared memory
  // access precedes it) and has published its block maximum
  cluster.sync();
  unsigned int E = 0u;
  for (int q = 0; q < CS; ++q) E = max(E, *cluster.map_shared_rank(eslot, q));
  // Exchange by push: when every CTA of the cluster holds a replica, each CTA
  // copies its new u slice, per consumer the part within the consumer's target
  // range, straight into the consumers' replicas (shared-to-shared bulk copies
  // completing on the consumer's rbar), instead of through L2 and a barrier.
  // Bounds are even (16-byte pairs); a slice ending at an odd N sends one pair
  // more, which lands past the last target the consumer reads.
  if (warp == 0) {
    int ok = 1;
    if (lane < CS) {
      const int* ri = cluster.map_shared_rank(rinfo, lane);
      cf0[lane] = ri[0]; cf1[lane] = ri[1]; croff[lane] = ri[2]; ok = ri[3];
    }
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) push_s = (!LOCAL && ok) ? 1 : 0;
  }
  __syncthreads();
  const bool push = push_s != 0;
  // bytes this CTA receives per exchange: the parts of every slice in [f0, f1)
  unsigned int push_expect = 0u;
  if (push)
    for (int q = 0; q < CS; ++q) {
      const int s0 = max(sbound[q], f0), e1 = (min(sbound[q + 1], f1) + 1) & ~1;
      if (e1 > s0) push_expect += 8u * (unsigned int)(e1 - s0);
    }
  const int shift = (int)E - 1023;                  // max |rhs| 2^-shift in [1, 2)
  // r0 = rhs (scaled) and x0 = 0 for the first pass
  for (int k = tid; k < nl; k += PINS_DDCG_TPB) {
    rv[k] = split_f64(rhs_of(lo + k), shift);
    xv[k] = make_float2(0.f, 0.f);
  }
  __syncthreads();                                  // rb[], entries visible in the block
  int t0 = 0;                                       // last local unknown with rb <= c0
  if (c0 < c1) {
    int lo_s = 0, hi_s = nl - 1;
    while (lo_s < hi_s) {
      const int mid = (lo_s + hi_s + 1) >> 1;
      if (rb[mid] <= c0) lo_s = mid; else hi_s = mid - 1;
    }
    t0 = lo_s;
  }
  const bool starts_mid = (c0 < c1) && rb[t0] < c0;
  // The slice structure is fixed for the launch: a row cut by this slice's
  // start is its head (hrow), a row cut by its end its tail.  A tail is
  // completed from the heads of the following slices up to run_end (empty
  // slices, hrow = -2, contribute zero).
  const int lastrow = (c0 < c1) ? erow[(c1 - 1 - c0) * PINS_DDCG_TPB + tid] : -1;
  const int firstrow = (c0 < c1) ? erow[tid] : -1;
  const bool single_run = (c0 < c1) && firstrow == lastrow;
  const bool is_tail = (c0 < c1) && rb[lastrow + 1] > c1 && !(single_run && starts_mid);
  hrow[tid] = (c0 < c1) ? (starts_mid ? firstrow : -1) : -2;
  __syncthreads();
  int run_end = tid;
  if (is_tail)
    for (int k = tid + 1; k < PINS_DDCG_TPB; ++k) {
      if (hrow[k] == -2) continue;
      if (hrow[k] != lastrow) break;
      run_end = k;
    }

  // od[t] = sum over the row/column entries of (S/eta) u, for the own unknowns.
  // Products first (independent), then a sum over runs of equal local row; a
  // row cut by the slice start is this thread's head, a row cut by its end its
  // tail (completed below from the following threads' heads, in thread order).
  auto spmv = [&](const float2* src, const float2* lsrc, bool sm) {
    float2 headv = make_float2(0.f, 0.f), tailv = make_float2(0.f, 0.f);
    int headrow = -1, tailrow = -1;
    if (c0 < c1) {
      int cur = firstrow;
      bool first = true;
      float2 acc = make_float2(0.f, 0.f);
      for (int base = c0; base < c1; base += 4) {
        int tg[4], rw[4]; float2 v[4], uu[4]; float ph[4], pl[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const bool ok = base + q < c1;
          const int sl = (base + q - c0) * PINS_DDCG_TPB + tid;
          tg[q] = ok ? etg[sl] : 0;
          v[q] = ok ? eva[sl] : make_float2(0.f, 0.f);
          rw[q] = ok ? erow[sl] : cur;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) uu[q] = sm ? lsrc[tg[q]] : __ldcg(src + tg[q]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          two_prod(v[q].x, uu[q].x, ph[q], pl[q]);
          pl[q] = __fmaf_rn(v[q].x, uu[q].y, __fmaf_rn(v[q].y, uu[q].x, pl[q]));
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (base + q < c1) {
            if (rw[q] != cur) {                     // row cur ended inside the slice
              if (first && starts_mid) { headrow = cur; headv = acc; }
              else od[cur] = acc;
              first = false;
              acc = make_float2(0.f, 0.f);
              cur = rw[q];
            }
            float t1, t2; two_sum(acc.x, ph[q], t1, t2);
            acc.x = t1; acc.y = __fadd_rn(acc.y, __fadd_rn(t2, pl[q]));
          }
        }
      }
      if (first && starts_mid) { headrow = cur; headv = acc; }
      else if (rb[cur + 1] > c1) { tailrow = cur; tailv = acc; }
      else od[cur] = acc;
    }
    (void)headrow;
    hval[tid] = headv;                              // zero for an empty slice or no head
    __syncthreads();
    if (tailrow >= 0) {
      // heads of the following slices, four independent partial sums
      float2 s0 = tailv, s1 = make_float2(0.f, 0.f), s2 = s1, s3 = s1;
      int k = tid + 1;
      for (; k + 3 <= run_end; k += 4) {
        s0 = ddv_add(s0, hval[k]);
        s1 = ddv_add(s1, hval[k + 1]);
        s2 = ddv_add(s2, hval[k + 2]);
        s3 = ddv_add(s3, hval[k + 3]);
      }
      for (; k <= run_end; ++k) s0 = ddv_add(s0, hval[k]);
      od[tailrow] = ddv_add(ddv_add(s0, s1), ddv_add(s2, s3));
    }
    __syncthreads();
  };
  // three block partials (double-float) -> slot buffer `b` of every CTA (the
  // cluster barrier that follows publishes them)
  auto shfl2 = [](float2 v, int o) -> float2 {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
  };
  auto warp_sum2 = [&](float2 v) -> float2 {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = ddv_add(v, shfl2(v, o));
    return v;
  };
  int CSP = 1;
  while (CSP < CS) CSP <<= 1;
  auto norm2 = [](float2 v) { float h, l; fast_two_sum(v.x, v.y, h, l); return make_float2(h, l); };
  auto publish3 = [&](float2 v0, float2 v1, float2 v2, int b) {
    v0 = warp_sum2(norm2(v0)); v1 = warp_sum2(norm2(v1)); v2 = warp_sum2(norm2(v2));
    if (lane == 0) { red[0][warp] = v0; red[1][warp] = v1; red[2][warp] = v2; }
    __syncthreads();
    if (warp == 0) {
      // every group of W lanes holds the W warp partials: after log2(W)
      // butterfly levels every lane holds the same block total
      constexpr int W = PINS_DDCG_TPB / 32;
      float2 b0 = red[0][lane & (W - 1)], b1 = red[1][lane & (W - 1)], b2 = red[2][lane & (W - 1)];
#pragma unroll
      for (int o = W / 2; o > 0; o >>= 1) {
        b0 = ddv_add(b0, shfl2(b0, o));
        b1 = ddv_add(b1, shfl2(b1, o));
        b2 = ddv_add(b2, shfl2(b2, o));
      }
      if (lane < CS) {
        float2* rs = cluster.map_shared_rank(&slot[b][0][0], lane);
        rs[0 * PINS_DDCG_MAX + rank] = b0;
        rs[1 * PINS_DDCG_MAX + rank] = b1;
        rs[2 * PINS_DDCG_MAX + rank] = b2;
      }
    }
  };
  // every warp sums the slots of buffer `b` in the same butterfly order
  // (bit-identical in all lanes and CTAs) and converts the totals to FP64
  // (every group of CSP lanes, CSP the power of two >= CS, holds the CS slots
  // and zeros, so log2(CSP) levels leave the same total in every lane)
  auto gather3 = [&](int b, float2& t0r, float2& t1r, float2& t2r) {
    const float2 z = make_float2(0.f, 0.f);
    const int sl = lane & (CSP - 1);
    float2 q0 = sl < CS ? slot[b][0][sl] : z;
    float2 q1 = sl < CS ? slot[b][1][sl] : z;
    float2 q2 = sl < CS ? slot[b][2][sl] : z;
    for (int o = CSP >> 1; o > 0; o >>= 1) {
      q0 = ddv_add(q0, shfl2(q0, o));
      q1 = ddv_add(q1, shfl2(q1, o));
      q2 = ddv_add(q2, shfl2(q2, o));
    }
    t0r = q0; t1r = q1; t2r = q2;
  };

  // acc += x y for double-float x, y, accumulated unnormalised (hi by TwoSum,
  // every lower-order term into lo); normalised once in the reductions below
  auto acc2 = [](float2& acc, float2 x, float2 y) {
    float p, e; two_prod(x.x, y.x, p, e);
    e = __fmaf_rn(x.x, y.y, __fmaf_rn(x.y, y.x, e));
    float sh, st; two_sum(acc.x, p, sh, st);
    acc.x = sh; acc.y = __fadd_rn(acc.y, __fadd_rn(st, e));
  };
  // a barrier over the cluster; a cluster of one needs only its block's
  auto csync = [&]() {
    if (LOCAL) __syncthreads(); else cluster.sync();
  };
  const float2 zero = make_float2(0.f, 0.f);
  // ur <- the exchange buffer src (after the barrier that published it): bulk
  // copies of up to 16 KB issued by thread 0, completed on rbar.  A wait that
  // gives up (flag bit 7) ends the replica for this launch: the CTA returns to
  // reading src through L2 and the caller poisons its partials, so that every
  // CTA leaves the iteration.
  bool rep_dead = false;
  // push: each thread's u stores are ordered before the copy engine reads them,
  // then lane c of warp 0 sends consumer c its part
  auto push_out = [&]() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid < CS) {
      const int c = tid;
      const int s0 = max(lo, cf0[c]), e1 = (min(lo + nl, cf1[c]) + 1) & ~1;
      if (e1 > s0) {
        const unsigned int dst = ddcg_mapa(ddcg_smem + croff[c] + 8 * (s0 - cf0[c]), (unsigned)c);
        const unsigned int bar = ddcg_mapa(&rbar, (unsigned)c);
        asm volatile(
            "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
            ::"r"(dst), "r"(smem_u32(uv + (s0 - lo))), "r"(8u * (unsigned int)(e1 - s0)), "r"(bar)
            : "memory");
      }
    }
  };
  // push: wait until every part of this exchange has arrived (bounded; a wait
  // that gives up sets flag bit 7 and the caller poisons its partials)
  auto push_in = [&]() -> bool {
    if (tid == 0) mbar_expect_tx(&rbar, push_expect);
    const bool ok = __syncthreads_and(mbar_wait_bounded(&rbar, rpar, 1u << 22));
    if (ok) { rpar ^= 1u; return true; }
    if (tid == 0) atomicOr(a.flag, 128);
    rep_dead = true;
    return false;
  };
  auto fetch = [&](const float2* src) -> bool {
    if (tid == 0) {
      asm volatile("fence.proxy.async;" ::: "memory");
      mbar_expect_tx(&rbar, rep_bytes);
      for (unsigned int off = 0; off < rep_bytes; off += 16384u)
        bulk_g2s(reinterpret_cast<char*>(ur) + off, reinterpret_cast<const char*>(src) + off,
                 min(16384u, rep_bytes - off), &rbar);
    }
    const bool ok = __syncthreads_and(mbar_wait_bounded(&rbar, rpar, 1u << 22));
    if (ok) { rpar ^= 1u; return true; }
    if (tid == 0) atomicOr(a.flag, 128);
    rep = false;
    rep_dead = true;
    return false;
  };

  // Passes: PCG from (x, r) until the recurrence residual meets the tolerance;
  // then the true residual rhs - M x is formed (one more exchange and SpMV).  If
  // it is above twice the tolerance -- the recurrences of a long run can drift
  // from it -- the next pass restarts from x with r = rhs - M x.  The scalar
  // recurrences run in double-float on the FP32 units: FP64 on this GPU issues
  // at ~1/64 of the FP32 rate and every thread forms the scalars.
  const float tol2 = (float)a.rtol2;
  float2 bb = zero, rr = zero;
  int it = 0, sb = 0;                               // sb: slot set of the next publish
  bool conv = false;
  for (int pass = 0; pass < PINS_DDCG_PASSES; ++pass) {
    // u0 = D^-1 r0 published; p = s = 0 (the first step takes beta = 0)
    for (int k = tid; k < nl; k += PINS_DDCG_TPB) {
      const float2 u0 = ddv_scale(dinv[k], rv[k]);
      uv[k] = u0;
      sv[k] = zero;
      pv[k] = zero;
      if (!LOCAL && !push) __stcg(ug0 + lo + k, u0);
    }
    // the generic-proxy stores above are read by other CTAs' bulk copies
    if (push) push_out();
    else if (!LOCAL) asm volatile("fence.proxy.async.global;" ::: "memory");
    float2 rgam_prev = make_float2(1.f, 0.f), ralp_prev = rgam_prev;
    int itr = 0;
    conv = false;
    while (true) {
      bool poison = false;
      if (push) {
        poison = rep_dead || !push_in();            // every part of u in the replica
      } else {
        csync();                                    // every u slice published
        if (rep) poison = !fetch(ug0 + f0);
      }
      spmv(ug0 + f0, LOCAL ? uv : ur, LOCAL || rep);
      // w = M u of the own unknowns and the (r.u, w.u, r.r) partials
      float2 lg = zero, ld = zero, lrr = zero;
      for (int k = tid; k < nl; k += PINS_DDCG_TPB) {
        const float2 uk = uv[k], rk = rv[k];
        const float2 w = ddv_add(ddv_mul(dg[k], uk), od[k]);
        wv[k] = w;
        od[k] = zero;
        acc2(lg, rk, uk);
        acc2(ld, w, uk);
        acc2(lrr, rk, rk);
      }
      if (poison) lrr = make_float2(__int_as_float(0x7fc00000), 0.f);
      publish3(lg, ld, lrr, sb);
      csync();                                      // partials published
      // scalars (identical in every CTA)
      float2 gam, dlt;
      gather3(sb, gam, dlt, rr);
      sb ^= 1;
      if (pass == 0 && itr == 0) bb = rr;
      if (!(bb.x > 0.f)) break;
      if (!(rr.x > tol2 * bb.x)) { conv = true; break; }
      if (!(rr.x == rr.x) || it >= a.max_iter) break;   // NaN or the cap stops
      // beta = gam / gam', alpha = gam / (dlt - beta gam / alpha'); the
      // difference can cancel, so it is formed in double-float.  1/gam' and
      // 1/alpha' were formed in the previous iteration, off this path.
      const float2 beta = (itr == 0) ? zero : ddv_mul(gam, rgam_prev);
      const float2 den = (itr == 0) ? dlt
                                    : ddv_add(dlt, ddv_neg(ddv_mul(ddv_mul(beta, gam), ralp_prev)));
      const float2 alpha = ddv_div(gam, den);
      const float2 nalpha = ddv_neg(alpha);
      // p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = D^-1 r,
      // with double-float step lengths: rounding them to FP32 (relative 2^-24
      // per step) costs conjugacy fast enough that these systems stall
      for (int k = tid; k < nl; k += PINS_DDCG_TPB) {
        const float2 pk = ddv_axpy2(beta, pv[k], uv[k]);
        const float2 sk = ddv_axpy2(beta, sv[k], wv[k]);
        const float2 xk = ddv_axpy2(alpha, pk, xv[k]);
        const float2 rk = ddv_axpy2(nalpha, sk, rv[k]);
        const float2 uk = ddv_scale(dinv[k], rk);
        pv[k] = pk; sv[k] = sk; xv[k] = xk; rv[k] = rk; uv[k] = uk;
        if (!LOCAL && !push) __stcg(ug0 + lo + k, uk);
      }
      if (push) push_out();
      else if (!LOCAL) asm volatile("fence.proxy.async.global;" ::: "memory");
      // the next step's 1/gam' and 1/alpha', formed while the exchange is in flight
      rgam_prev = ddv_div(make_float2(1.f, 0.f), gam);
      ralp_prev = ddv_div(make_float2(1.f, 0.f), alpha);
      ++it;
      ++itr;
    }
    if (!conv || pass + 1 == PINS_DDCG_PASSES) break;
    // true residual t = rhs - M x: x goes through its own exchange buffer, last
    // read before the barrier of the previous pass's check
    if (!LOCAL)
      for (int k = tid; k < nl; k += PINS_DDCG_TPB) __stcg(ug1 + lo + k, xv[k]);
    csync();                                        // x slices published
    spmv(ug1 + f0, xv, LOCAL);
    float2 lt = zero;
    for (int k = tid; k < nl; k += PINS_DDCG_TPB) {
      const float2 mx = ddv_add(ddv_mul(dg[k], xv[k]), od[k]);
      od[k] = zero;
      const float2 t = ddv_add(split_f64(rhs_of(lo + k), shift), make_float2(-mx.x, -mx.y));
      rv[k] = t;
      acc2(lt, t, t);
    }
    publish3(lt, zero, zero, sb);
    csync();
    float2 tt, d1, d2;
    gather3(sb, tt, d1, d2);
    sb ^= 1;
    rr = tt;
    if (!(tt.x > 4.f * tol2 * bb.x)) break;         // within twice the tolerance
    conv = false;
  }
  // a replica copy left in flight by a wait that gave up is awaited (bounded)
  // before the CTA's shared memory goes away
  if (rep_dead) mbar_wait_bounded(&rbar, rpar, 1u << 22);
  const double scale = ldexp(1.0, shift);
  double dg0 = 0.0, dg1 = 0.0;                      // <rhs, x>, <ab, x> partials
  for (int k = tid; k < nl; k += PINS_DDCG_TPB) {
    const double xk = ((double)xv[k].x + (double)xv[k].y) * scale;
    a.x[lo + k] = xk;
    if (a.dots) { dg0 += rhs_of(lo + k) * xk; dg1 += a.ab[lo + k] * xk; }
  }
  if (a.dots) {   // block sums in a fixed tree, then rank 0 adds the CTAs in rank order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dg0 += __shfl_xor_sync(0xffffffffu, dg0, o);
      dg1 += __shfl_xor_sync(0xffffffffu, dg1, o);
    }
    if (lane == 0) { dred[0][warp] = dg0; dred[1][warp] = dg1; }
    __syncthreads();
    if (tid == 0) {
      double b0 = 0.0, b1 = 0.0;
      for (int w = 0; w < PINS_DDCG_TPB / 32; ++w) { b0 += dred[0][w]; b1 += dred[1][w]; }
      double* rs = cluster.map_shared_rank(&dslot[0][0], 0);
      rs[rank] = b0;
      rs[PINS_DDCG_MAX + rank] = b1;
    }
  }
  if (rank == 0 && tid == 0) {
    a.info[0] = (double)it;
    const double rrd = (double)rr.x + (double)rr.y, bbd = (double)bb.x + (double)bb.y;
    a.info[1] = (bbd > 0.0) ? sqrt(rrd / bbd) : 0.0;
  }
  cluster.sync();                                   // no CTA exits while others read its u
  if (a.dots && rank == 0 && tid == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int q = 0; q < CS; ++q) { t0 += dslot[0][q]; t1 += dslot[1][q]; }
    a.dots[0] = t0;
    a.dots[1] = t1;
  }
}

// largest cluster the device runs with this kernel's shared memory: 16 CTAs
// (non-portable size) where available, else 8; decided once, thread-safely, so
// that concurrent solves of one size always use the same cluster size
static int ddcg_max_cluster() {
  static const int cs = [] {
    cudaFuncSetAttribute(k_pcg_dd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         PINS_DDCG_SMEM);
    cudaFuncSetAttribute(k_pcg_dd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         PINS_DDCG_SMEM);
    int v = 8;
    if (cudaFuncSetAttribute(k_pcg_dd<false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
        cudaSuccess) {
      cudaLaunchConfig_t lc = {};
      lc.gridDim = dim3(16);
      lc.blockDim = dim3(PINS_DDCG_TPB);
      lc.dynamicSmemBytes = PINS_DDCG_SMEM;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 16; attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
      lc.attrs = attr; lc.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, k_pcg_dd<false>, &lc) == cudaSuccess &&
          nclusters >= 1)
        v = 16;
    }
    cudaGetLastError();
    return v;
  }();
  return cs;
}

size_t ddcg_smem_bytes(int N, int cs) {
  const int L4 = (ddcg_slice_cap(N, cs) + 3) & ~3;
  return (size_t)PINS_DDCG_PER_UNKNOWN * L4 + 16;
}

// cluster size for N unknowns (a power of two up to maxcs), with at least as
// many CTAs as the shared memory needs
static int ddcg_cluster_for(int N, int maxcs) {
  if (N <= PINS_DDCG_LOCAL_MAX && ddcg_smem_bytes(N, 1) <= PINS_DDCG_SMEM) return 1;
  int cs = 2;
  while (cs < maxcs && ((N + cs - 1) / cs > PINS_DDCG_SLICE ||
                        ddcg_smem_bytes(N, cs) > PINS_DDCG_SMEM))
    cs *= 2;
  return cs;
}

cudaError_t launch_pcg_dd(int m, int n, double eta, const double* r, const double* c,
                          const int* indptr, const int* indices, const double* data,
                          const int* colptr, const int* rowidx, const double* cdata,
                          const double* rhs, double* x, const double* ab, double* dots,
                          int* ent_tgt, float2* ent_val, int* ent_row, float* ug, int nnz,
                          double rtol, int max_iter, double* info, int* flag, cudaStream_t st,
                          bool* used) {
  *used = false;
  const int N = m + n;
  const int CS = ddcg_cluster_for(N, ddcg_max_cluster());
  const int L = ddcg_slice_cap(N, CS);
  if (ddcg_smem_bytes(N, CS) > PINS_DDCG_SMEM || L > 0xffff) return cudaSuccess;   // caller falls back
  // dynamic shared memory: the slice, room for the entries (1.5x the even share
  // plus 512) and, in a cluster, for a replica of half the unknowns -- not the
  // whole allocation, so that CTAs of other kernels can share these SMs.  A CTA
  // whose entries or replica do not fit reads them from global memory.
  size_t smem = ddcg_smem_bytes(N, CS);
  const size_t share = (size_t)2 * (size_t)(nnz > 0 ? nnz : 0) / (size_t)CS;
  smem += (size_t)16 * ((share + share / 2 + 512 + PINS_DDCG_TPB - 1) / PINS_DDCG_TPB * PINS_DDCG_TPB);
  if (CS > 1) smem += (size_t)8 * ((size_t)N / 2 + 64);
  smem = std::min(smem, (size_t)PINS_DDCG_SMEM);
  CGddArgs a;
  a.m = m; a.n = n; a.inv_eta = 1.0 / eta;
  a.r = r; a.c = c; a.indptr = indptr; a.indices = indices; a.data = data;
  a.colptr = colptr; a.rowidx = rowidx; a.cdata = cdata;
  a.rhs = rhs; a.x = x; a.ab = ab; a.dots = dots;
  a.ent_tgt = ent_tgt; a.ent_val = ent_val; a.ent_row = ent_row;
  a.ug = ug;
  a.smem_bytes = smem;
  a.rtol2 = rtol * rtol; a.max_iter = max_iter; a.info = info; a.flag = flag;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(CS);
  lc.blockDim = dim3(PINS_DDCG_TPB);
  lc.dynamicSmemBytes = smem;
  lc.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS; attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  *used = true;
  return CS == 1 ? cudaLaunchKernelEx(&lc, k_pcg_dd<true>, a)
                 : cudaLaunchKernelEx(&lc, k_pcg_dd<false>, a);
}

}  // namespace pins
