// Truncated Jacobi-preconditioned CG of the Newton step (Algorithm 2), run by one
// thread-block cluster with every vector resident in shared memory.
//
// Ordering: the single-reduction form of PCG (Chronopoulos & Gear, J. Comput.
// Appl. Math. 25, 1989): per iteration one matrix-vector product w = M u with
// u = D^-1 r and one fused reduction of (r.u, w.u, r.r); the recurrences
//   x += alpha p,  r -= alpha s,  u = D^-1 r,  w = M u,
//   beta = g'/g,  alpha = g'/(d' - beta g'/alpha),  p = u + beta p,  s = w + beta s
// give the same iterates as the textbook Jacobi PCG in exact arithmetic, with the
// same stopping rule (||r|| <= rtol ||rhs||) and the same iteration count.
//
// Layout: CTA `rank` owns unknowns [rank L, rank L + L) and keeps u, r, x, p, s,
// w and D^-1 for them in shared memory; the SpMV reads other CTAs' u through
// distributed shared memory.  Each CTA reduces its three partials, stores them
// into a slot of every CTA (DSMEM stores), and after one cluster barrier every
// CTA sums the slots in the same tree order, so all CTAs take identical,
// reproducible decisions.  Two cluster barriers per iteration.
#include <cooperative_groups.h>
#include "pins_kernels.h"

namespace cg = cooperative_groups;

namespace pins {

#define PINS_CGC_MAX 16
#define PINS_CGC_TPB 256
#define PINS_CGC_ARRAYS 8

struct CGClusterArgs {
  int m, n; double inv_eta;
  const double* r; const double* c;
  const int* indptr; const int* indices; const double* data;
  const int* colptr; const int* rowidx; const double* cdata;
  const double* rhs; double* x;
  double rtol2; int max_iter; double* info;
  int* flag;        // set (bit 1/2) if an index fell outside the cluster's slices
};

__global__ void __launch_bounds__(PINS_CGC_TPB) k_pcg_cg1(CGClusterArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double cg1_smem[];
  __shared__ double* rem[PINS_CGC_MAX];
  __shared__ double slot[3 * PINS_CGC_MAX];
  __shared__ double red[3][PINS_CGC_TPB / 32];
  __shared__ double bc[8];
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int N = a.m + a.n;
  const int L = (N + CS - 1) / CS;
  const int lo = rank * L;
  const int nl = max(0, min(N, lo + L) - lo);
  double* u = cg1_smem;            // remotely read
  double* rv = u + L;
  double* xv = rv + L;
  double* pv = xv + L;
  double* sv = pv + L;
  double* wv = sv + L;
  double* dv = wv + L;
  double* od = dv + L;             // off-diagonal part of M u
  __shared__ int hrow[PINS_CGC_TPB];
  __shared__ double hval[PINS_CGC_TPB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < CS) rem[tid] = cluster.map_shared_rank(u, tid);

  // Off-diagonal part of M u, balanced by entries.  The CSR rows (unknowns
  // t < m) and CSC columns (t >= m) form one entry space: unknown t owns
  // entries [beg(t), beg(t + 1)).  Each thread takes an equal slice of this
  // CTA's entries; a row split between threads is summed by the thread holding
  // its first entry, adding the following threads' pieces in thread order.
  const int Kc = __ldg(a.indptr + a.m);
  auto beg = [&](int t) -> int {
    return (t < a.m) ? __ldg(a.indptr + t) : Kc + __ldg(a.colptr + t - a.m);
  };
  auto entry = [&](int e, double& v) -> int {   // target unknown, value
    if (e < Kc) { v = __ldg(a.data + e); return a.m + __ldg(a.indices + e); }
    v = __ldg(a.cdata + e - Kc); return __ldg(a.rowidx + e - Kc);
  };
  const int E0 = beg(min(lo, N)), E1 = beg(min(lo + nl, N));
  const int c0 = E0 + (int)(((long long)tid * (E1 - E0)) / PINS_CGC_TPB);
  const int c1 = E0 + (int)(((long long)(tid + 1) * (E1 - E0)) / PINS_CGC_TPB);
  int t0 = lo;                                      // unknown holding entry c0
  if (c0 < c1) {
    int lo_s = lo, hi_s = lo + nl - 1;              // largest t with beg(t) <= c0
    while (lo_s < hi_s) {
      const int mid = (lo_s + hi_s + 1) >> 1;
      if (beg(mid) <= c0) lo_s = mid; else hi_s = mid - 1;
    }
    t0 = lo_s;
  }
  auto spmv_all = [&]() {
    int t = t0, e = c0;
    bool head = (c0 < c1) && beg(t0) < c0;
    double acc = 0.0, head_val = 0.0, tail_val = 0.0;
    int head_row = -1, tail_row = -1;
    while (e < c1) {
      const int rend = beg(t + 1);
      const int se = min(rend, c1);
      for (; e < se; ++e) {
        double v;
        const int g = entry(e, v);
        const int ow = g / L;
        if ((unsigned)ow >= (unsigned)CS || (unsigned)(g - ow * L) >= (unsigned)L) {
          atomicOr(a.flag, 1); continue;
        }
        acc += v * rem[ow][g - ow * L];
      }
      if (head) { head_val = acc; head_row = t; head = false; }
      else if (rend <= c1) { od[t - lo] = acc; }
      else { tail_val = acc; tail_row = t; }
      acc = 0.0;
      if (rend <= c1) ++t;
    }
    hrow[tid] = (c0 < c1) ? head_row : -2;          // -2: empty slice, skipped below
    hval[tid] = head_val;
    __syncthreads();
    if (tail_row >= 0) {
      double s = tail_val;
      for (int k = tid + 1; k < PINS_CGC_TPB; ++k) {
        if (hrow[k] == -2) continue;
        if (hrow[k] != tail_row) break;
        s += hval[k];
      }
      od[tail_row - lo] = s;
    }
    __syncthreads();
  };
  // (M u)_t for the own unknowns, after spmv_all
  auto mrow = [&](int k) -> double {
    const int t = lo + k;
    const double d = (t < a.m) ? __ldg(a.r + t) : __ldg(a.c + t - a.m);
    return (d * u[k] + od[k]) * a.inv_eta;
  };
  // block partials of three dot products -> every CTA's slots -> cluster barrier
  // -> tree sum in warp 0 (same order in every CTA); totals land in bc[0..2]
  auto reduce3 = [&](double v0, double v1, double v2) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v0 += __shfl_xor_sync(0xffffffffu, v0, o);
      v1 += __shfl_xor_sync(0xffffffffu, v1, o);
      v2 += __shfl_xor_sync(0xffffffffu, v2, o);
    }
    if (lane == 0) { red[0][warp] = v0; red[1][warp] = v1; red[2][warp] = v2; }
    __syncthreads();
    if (warp == 0) {
      constexpr int W = PINS_CGC_TPB / 32;
      double b0 = lane < W ? red[0][lane] : 0.0;
      double b1 = lane < W ? red[1][lane] : 0.0;
      double b2 = lane < W ? red[2][lane] : 0.0;
      // full butterfly: every lane (each stores into one CTA below) holds the
      // block total, so all CTAs receive the same partial
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        b0 += __shfl_xor_sync(0xffffffffu, b0, o);
        b1 += __shfl_xor_sync(0xffffffffu, b1, o);
        b2 += __shfl_xor_sync(0xffffffffu, b2, o);
      }
      if (lane < CS) {
        double* rs = cluster.map_shared_rank(slot, lane);
        rs[0 * CS + rank] = b0;
        rs[1 * CS + rank] = b1;
        rs[2 * CS + rank] = b2;
      }
    }
    cluster.sync();
    if (warp == 0) {
      double t0 = lane < CS ? slot[0 * CS + lane] : 0.0;
      double t1 = lane < CS ? slot[1 * CS + lane] : 0.0;
      double t2 = lane < CS ? slot[2 * CS + lane] : 0.0;
#pragma unroll
      for (int o = PINS_CGC_MAX / 2; o > 0; o >>= 1) {
        t0 += __shfl_xor_sync(0xffffffffu, t0, o);
        t1 += __shfl_xor_sync(0xffffffffu, t1, o);
        t2 += __shfl_xor_sync(0xffffffffu, t2, o);
      }
      if (lane == 0) { bc[0] = t0; bc[1] = t1; bc[2] = t2; }
    }
    __syncthreads();
  };

  // x = 0, r = rhs, u = D^-1 r
  for (int k = tid; k < nl; k += PINS_CGC_TPB) {
    const int t = lo + k;
    const double d = (t < a.m) ? __ldg(a.r + t) : __ldg(a.c + t - a.m);
    const double di = 1.0 / (d * a.inv_eta);
    const double r0 = a.rhs[t];
    dv[k] = di; rv[k] = r0; xv[k] = 0.0; u[k] = di * r0; od[k] = 0.0;
  }
  cluster.sync();                                   // rem[] and every u slice ready
  spmv_all();
  double lg = 0.0, ld = 0.0, lr = 0.0;
  for (int k = tid; k < nl; k += PINS_CGC_TPB) {
    const double w = mrow(k);
    wv[k] = w; pv[k] = u[k]; sv[k] = w;
    lg += rv[k] * u[k]; ld += w * u[k]; lr += rv[k] * rv[k];
  }
  reduce3(lg, ld, lr);
  const double bb = bc[2];
  // the scalar recurrence runs in thread 0 only and is broadcast through bc[]
  double gam = bc[0], alpha_s = (bc[1] != 0.0) ? bc[0] / bc[1] : 0.0;
  double alpha = alpha_s;
  int it = 0;
  double rr = bb;
  if (bb > 0.0) {
    while (it < a.max_iter) {
      for (int k = tid; k < nl; k += PINS_CGC_TPB) {
        xv[k] += alpha * pv[k];
        const double r1 = rv[k] - alpha * sv[k];
        rv[k] = r1;
        u[k] = dv[k] * r1;
      }
      ++it;
      cluster.sync();                               // every u slice updated
      spmv_all();
      lg = 0.0; ld = 0.0; lr = 0.0;
      for (int k = tid; k < nl; k += PINS_CGC_TPB) {
        const double w = mrow(k);
        wv[k] = w;
        lg += rv[k] * u[k]; ld += w * u[k]; lr += rv[k] * rv[k];
      }
      reduce3(lg, ld, lr);
      rr = bc[2];
      if (tid == 0) {
        const bool stop = !(rr > a.rtol2 * bb);    // ||r|| <= rtol ||rhs|| (NaN stops)
        double beta_s = 0.0;
        if (!stop) {
          const double gn = bc[0];
          beta_s = gn / gam;
          alpha_s = gn / (bc[1] - beta_s * gn / alpha_s);
          gam = gn;
        }
        bc[3] = stop ? 1.0 : 0.0; bc[4] = beta_s; bc[5] = alpha_s;
      }
      __syncthreads();
      if (bc[3] != 0.0) break;
      const double beta = bc[4];
      alpha = bc[5];
      for (int k = tid; k < nl; k += PINS_CGC_TPB) {
        pv[k] = u[k] + beta * pv[k];
        sv[k] = wv[k] + beta * sv[k];
      }
      // the next iteration rewrites u only after every CTA has read it in this
      // iteration's SpMV: the reduce3 barrier above orders them
    }
  }
  for (int k = tid; k < nl; k += PINS_CGC_TPB) a.x[lo + k] = xv[k];
  if (rank == 0 && tid == 0) {
    a.info[0] = (double)it;
    a.info[1] = (bb > 0.0) ? sqrt(rr / bb) : 0.0;
  }
  cluster.sync();                                   // no CTA exits while others read its u
}

// 16 CTAs (non-portable cluster size) where the device runs them with this
// kernel's shared memory, else 8; decided once, thread-safely
static int cg1_cluster_size() {
  static const int cs = [] {
    cudaFuncSetAttribute(k_pcg_cg1, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    int v = 8;
    if (cudaFuncSetAttribute(k_pcg_cg1, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
        cudaSuccess) {
      cudaLaunchConfig_t lc = {};
      lc.gridDim = dim3(16);
      lc.blockDim = dim3(PINS_CGC_TPB);
      lc.dynamicSmemBytes = 200 * 1024;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 16; attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
      lc.attrs = attr; lc.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, k_pcg_cg1, &lc) == cudaSuccess &&
          nclusters >= 1)
        v = 16;
    }
    cudaGetLastError();
    return v;
  }();
  return cs;
}

cudaError_t launch_pcg_cluster(int m, int n, double eta, const double* r, const double* c,
                               const int* indptr, const int* indices, const double* data,
                               const int* colptr, const int* rowidx, const double* cdata,
                               const double* rhs, double* x, double rtol, int max_iter,
                               double* info, int* flag, cudaStream_t st, bool* used) {
  *used = false;
  const int N = m + n;
  const int CS = cg1_cluster_size();
  const int L = (N + CS - 1) / CS;
  const size_t smem = sizeof(double) * (size_t)L * PINS_CGC_ARRAYS;
  if (smem > 200 * 1024) return cudaSuccess;        // too large: caller falls back
  CGClusterArgs a;
  a.m = m; a.n = n; a.inv_eta = 1.0 / eta;
  a.r = r; a.c = c; a.indptr = indptr; a.indices = indices; a.data = data;
  a.colptr = colptr; a.rowidx = rowidx; a.cdata = cdata;
  a.rhs = rhs; a.x = x; a.rtol2 = rtol * rtol; a.max_iter = max_iter; a.info = info;
  a.flag = flag;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(CS);
  lc.blockDim = dim3(PINS_CGC_TPB);
  lc.dynamicSmemBytes = smem;
  lc.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS; attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  *used = true;
  return cudaLaunchKernelEx(&lc, k_pcg_cg1, a);
}

}  // namespace pins
