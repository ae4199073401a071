// Sparse side of the Newton step (Algorithm 2): CSC assembly of the kept
// coupling entries, the truncated Jacobi-preconditioned CG on
//   M d = rhs,   M = (1/eta) [[diag r, S], [S^T, diag c]],
// and the O(m + n) vector kernels of the solver (FP64).
//
// FP64 on GB300 runs at ~1/64 of the FP32 rate (~19 SM-cycles per warp-wide FP64
// instruction), so scalar bookkeeping is done by one thread and broadcast, and the
// vector work is spread over a thread-block cluster.
#include <algorithm>
#include <cooperative_groups.h>
#include "pins_kernels.h"

namespace cg = cooperative_groups;

namespace pins {

// exclusive scan of cnt[0..len) into ptr[0..len], resets cnt to 0.  One CTA:
// each thread owns a contiguous chunk, chunk totals are scanned with warp
// shuffles, then every chunk is written from its offset.
__global__ void __launch_bounds__(1024) k_scan(int* cnt, int* ptr, int len) {
  __shared__ int wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (len + 1023) / 1024;
  const int b0 = min(len, tid * per), b1 = min(len, b0 + per);
  int tot = 0;
  for (int t = b0; t < b1; ++t) tot += cnt[t];
  int inc = tot;                                   // inclusive scan within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int w = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += v;
    }
    wsum[lane] = w;                                // inclusive warp totals
  }
  __syncthreads();
  int run = inc - tot + (warp > 0 ? wsum[warp - 1] : 0);
  for (int t = b0; t < b1; ++t) { const int v = cnt[t]; ptr[t] = run; run += v; cnt[t] = 0; }
  if (tid == 1023) ptr[len] = wsum[31];
}
void launch_scan(int* cnt, int* ptr, int len, cudaStream_t st) {
  k_scan<<<1, 1024, 0, st>>>(cnt, ptr, len);
}

// ------------------------------------------------------------------------- //
// CSC from the row-ordered CSR, in four launches: column counts (atomics),
// exclusive scan (colptr; the counts are reset), placement (an atomic slot per
// entry, so the order inside a column depends on timing), then every column's
// entries sorted by row (a warp per column).  Rows are unique within a column,
// so the result is the same on every run.  colcnt is zero on entry and on exit.
// ------------------------------------------------------------------------- //
__global__ void k_csc_count(const int* indptr, const int* indices, int m, int* colcnt) {
  const int K = indptr[m];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K; e += gridDim.x * blockDim.x)
    atomicAdd(colcnt + indices[e], 1);
}
__global__ void k_csc_place(const int* indptr, const int* indices, const double* data, int m,
                            const int* colptr, int* fill, int* trow, double* tval) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    for (int e = indptr[i]; e < indptr[i + 1]; ++e) {
      const int j = indices[e];
      const int pos = colptr[j] + atomicAdd(fill + j, 1);
      trow[pos] = i;
      tval[pos] = data[e];
    }
}
// Bitonic sort of up to 32 W (key, value) pairs held W per lane, virtual
// position p = w * 32 + lane, ascending by key.  Partners closer than 32 are in
// other lanes (shuffles), farther ones in another register slot of the same lane.
template <int W>
__device__ __forceinline__ void warp_bitonic(int (&r)[W], double (&v)[W]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32 * W; k <<= 1) {
#pragma unroll
    for (int h = k >> 1; h > 0; h >>= 1) {
      if (h >= 32) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
          const int w2 = w ^ (h >> 5);
          if (w2 > w) {
            const bool up = ((w * 32 + lane) & k) == 0;
            if (up ? r[w] > r[w2] : r[w] < r[w2]) {
              const int tr = r[w]; r[w] = r[w2]; r[w2] = tr;
              const double tv = v[w]; v[w] = v[w2]; v[w2] = tv;
            }
          }
        }
      } else {
#pragma unroll
        for (int w = 0; w < W; ++w) {
          const int rk = __shfl_xor_sync(0xffffffffu, r[w], h);
          const double vk = __shfl_xor_sync(0xffffffffu, v[w], h);
          const bool up = ((w * 32 + lane) & k) == 0, low = (lane & h) == 0;
          const bool take = low ? (up ? rk < r[w] : rk > r[w]) : (up ? rk > r[w] : rk < r[w]);
          if (take) { r[w] = rk; v[w] = vk; }
        }
      }
    }
  }
}
template <int W>
__device__ __forceinline__ void warp_sort_segment(int b, int len, const int* trow,
                                                  const double* tval, int* rowidx, double* cdata) {
  const int lane = threadIdx.x & 31;
  int r[W]; double v[W];
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const int q = w * 32 + lane;
    r[w] = (q < len) ? trow[b + q] : 0x7fffffff;
    v[w] = (q < len) ? tval[b + q] : 0.0;
  }
  if (len > 1) warp_bitonic<W>(r, v);
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const int q = w * 32 + lane;
    if (q < len) { rowidx[b + q] = r[w]; cdata[b + q] = v[w]; }
  }
}
// one warp sorts segment j of (trow, tval) by row into (rowidx, cdata); fill[j] = 0.
// Keys are unique within a segment, so the order is deterministic.  Segments
// longer than 128 entries are appended to a list (as `tag`) for k_long_segsort.
__device__ __forceinline__ void warp_seg_sort(int j, const int* ptr, int* fill, const int* trow,
                                              const double* tval, int* rowidx, double* cdata,
                                              int tag, int* longseg, int* nlong) {
  const int lane = threadIdx.x & 31;
  const int b = ptr[j], len = ptr[j + 1] - b;
  if (lane == 0) fill[j] = 0;
  if (len <= 32) warp_sort_segment<1>(b, len, trow, tval, rowidx, cdata);
  else if (len <= 64) warp_sort_segment<2>(b, len, trow, tval, rowidx, cdata);
  else if (len <= 128) warp_sort_segment<4>(b, len, trow, tval, rowidx, cdata);
  else if (lane == 0) longseg[atomicAdd(nlong, 1)] = tag;
}

// Long segments, one CTA each: a bitonic sort in shared memory for up to
// PINS_LONGSEG entries, rank counting above that.  tag < m: row tag of the CSR
// (by column); tag >= m: column tag - m of the CSC (by row).
#define PINS_LONGSEG 4096
__global__ void __launch_bounds__(1024)
k_long_segsort(const int* nlong, const int* longseg, int m, const int* indptr, const int* tcol,
               const double* tcval, int* indices, double* data, const int* colptr,
               const int* trow, const double* tval, int* rowidx, double* cdata) {
  extern __shared__ unsigned char lsm[];
  double* sv = reinterpret_cast<double*>(lsm);
  int* sk = reinterpret_cast<int*>(sv + PINS_LONGSEG);
  const int cnt = *nlong;
  for (int q = blockIdx.x; q < cnt; q += gridDim.x) {
    const int tag = longseg[q];
    const bool row = tag < m;
    const int* ptr = row ? indptr : colptr;
    const int id = row ? tag : tag - m;
    const int* tk = row ? tcol : trow;
    const double* tv = row ? tcval : tval;
    int* ok = row ? indices : rowidx;
    double* ov = row ? data : cdata;
    const int b = ptr[id], len = ptr[id + 1] - b;
    if (len <= PINS_LONGSEG) {
      int P2 = 1;
      while (P2 < len) P2 <<= 1;
      for (int t = threadIdx.x; t < P2; t += blockDim.x) {
        sk[t] = (t < len) ? tk[b + t] : 0x7fffffff;
        sv[t] = (t < len) ? tv[b + t] : 0.0;
      }
      __syncthreads();
      for (int k = 2; k <= P2; k <<= 1)
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
          for (int t = threadIdx.x; t < P2; t += blockDim.x) {
            const int l = t ^ jj;
            if (l > t) {
              const bool up = (t & k) == 0;
              if (up ? sk[t] > sk[l] : sk[t] < sk[l]) {
                const int x = sk[t]; sk[t] = sk[l]; sk[l] = x;
                const double y = sv[t]; sv[t] = sv[l]; sv[l] = y;
              }
            }
          }
          __syncthreads();
        }
      for (int t = threadIdx.x; t < len; t += blockDim.x) { ok[b + t] = sk[t]; ov[b + t] = sv[t]; }
      __syncthreads();
    } else {
      for (int t = threadIdx.x; t < len; t += blockDim.x) {
        const int r = tk[b + t];
        int rank = 0;
        for (int u = 0; u < len; ++u) rank += (tk[b + u] < r) ? 1 : 0;
        ok[b + rank] = r;
        ov[b + rank] = tv[b + t];
      }
    }
  }
}
__global__ void k_csc_segsort(const int* colptr, int m, int n, int* fill, const int* trow,
                              const double* tval, int* rowidx, double* cdata, int* longseg,
                              int* nlong) {
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += nw)
    warp_seg_sort(j, colptr, fill, trow, tval, rowidx, cdata, m + j, longseg, nlong);
}

// ------------------------------------------------------------------------- //
// CSR and CSC of the entries kept by the one-pass selection (FastSelState):
// counts per row and column, both scans, atomic placement, then a warp per row
// (by column) and per column (by row) sorts its segment.  Every kernel does
// nothing when the selection failed, so the previous CSR/CSC stay intact.
// ------------------------------------------------------------------------- //
__device__ __forceinline__ bool fast_kept(const FastSelState& f, float key, unsigned long long ij) {
  const unsigned int u = key_order(key), T = key_order(f.tau);
  return u > T || (u == T && ij <= f.tie_max);
}
__global__ void k_fast_count(const FastSelState* fs, const float* ckey,
                             const unsigned long long* cij, int* rowcnt, int* colcnt) {
  const FastSelState f = *fs;
  if (f.fail) return;
  for (unsigned int q = blockIdx.x * blockDim.x + threadIdx.x; q < f.ncand; q += gridDim.x * blockDim.x) {
    const unsigned long long ij = cij[q];
    if (fast_kept(f, ckey[q], ij)) {
      atomicAdd(rowcnt + (int)(ij >> 32), 1);
      atomicAdd(colcnt + (int)(ij & 0xffffffffu), 1);
    }
  }
}
// CTA 0 scans the row counts, CTA 1 the column counts (each as k_scan)
__global__ void __launch_bounds__(1024) k_scan2(const FastSelState* fs, int* c0, int* p0, int l0,
                                                int* c1, int* p1, int l1) {
  if (fs->fail) return;
  __shared__ int wsum[32];
  int* cnt = blockIdx.x ? c1 : c0;
  int* ptr = blockIdx.x ? p1 : p0;
  const int len = blockIdx.x ? l1 : l0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (len + 1023) / 1024;
  const int b0 = min(len, tid * per), b1 = min(len, b0 + per);
  int tot = 0;
  for (int t = b0; t < b1; ++t) tot += cnt[t];
  int inc = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int w = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += v;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  int run = inc - tot + (warp > 0 ? wsum[warp - 1] : 0);
  for (int t = b0; t < b1; ++t) { const int v = cnt[t]; ptr[t] = run; run += v; cnt[t] = 0; }
  if (tid == 1023) ptr[len] = wsum[31];
}
__global__ void k_fast_place(const FastSelState* fs, const float* ckey,
                             const unsigned long long* cij, const int* indptr, int* rowfill,
                             int* tcol, double* tcval, const int* colptr, int* colfill, int* trow,
                             double* tval) {
  const FastSelState f = *fs;
  if (f.fail) return;
  for (unsigned int q = blockIdx.x * blockDim.x + threadIdx.x; q < f.ncand; q += gridDim.x * blockDim.x) {
    const unsigned long long ij = cij[q];
    const float key = ckey[q];
    if (!fast_kept(f, key, ij)) continue;
    const int i = (int)(ij >> 32), j = (int)(ij & 0xffffffffu);
    const double v = exp((double)key);              // X~_ij from its FP32 log (mixed path)
    const int pr = indptr[i] + atomicAdd(rowfill + i, 1);
    tcol[pr] = j; tcval[pr] = v;
    const int pc = colptr[j] + atomicAdd(colfill + j, 1);
    trow[pc] = i; tval[pc] = v;
  }
}
__global__ void k_fast_segsort(const FastSelState* fs, int m, int n, const int* indptr,
                               int* rowfill, const int* tcol, const double* tcval, int* indices,
                               double* data, const int* colptr, int* colfill, const int* trow,
                               const double* tval, int* rowidx, double* cdata, int* longseg,
                               int* nlong) {
  if (fs->fail) return;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < m + n; s += nw) {
    if (s < m) warp_seg_sort(s, indptr, rowfill, tcol, tcval, indices, data, s, longseg, nlong);
    else warp_seg_sort(s - m, colptr, colfill, trow, tval, rowidx, cdata, s, longseg, nlong);
  }
}
static void launch_long_segsort(int m, const SparseWS& sw, cudaStream_t st) {
  static const bool configured = [] {
    cudaFuncSetAttribute(k_long_segsort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(PINS_LONGSEG * (sizeof(double) + sizeof(int))));
    return true;
  }();
  (void)configured;
  k_long_segsort<<<152, 1024, PINS_LONGSEG * (sizeof(double) + sizeof(int)), st>>>(
      sw.nlong, sw.longseg, m, sw.indptr, sw.tcol, sw.tcval, sw.indices, sw.data, sw.colptr,
      sw.trow, sw.tval, sw.rowidx, sw.cdata);
}

void build_sparse_from_candidates(const FastSelState* fs, const float* ckey,
                                  const unsigned long long* cij, int m, int n, int keep,
                                  const SparseWS& sw, cudaStream_t st) {
  const int cb = std::max(1, std::min((PINS_FAST_CAP + 255) / 256, 192));
  k_fast_count<<<cb, 256, 0, st>>>(fs, ckey, cij, sw.rowcnt, sw.colcnt);
  k_scan2<<<2, 1024, 0, st>>>(fs, sw.rowcnt, sw.indptr, m, sw.colcnt, sw.colptr, n);
  k_fast_place<<<cb, 256, 0, st>>>(fs, ckey, cij, sw.indptr, sw.rowcnt, sw.tcol, sw.tcval,
                                   sw.colptr, sw.colcnt, sw.trow, sw.tval);
  const int sb = std::max(1, std::min((m + n + 7) / 8, 2368));
  cudaMemsetAsync(sw.nlong, 0, sizeof(int), st);
  k_fast_segsort<<<sb, 256, 0, st>>>(fs, m, n, sw.indptr, sw.rowcnt, sw.tcol, sw.tcval,
                                     sw.indices, sw.data, sw.colptr, sw.colcnt, sw.trow, sw.tval,
                                     sw.rowidx, sw.cdata, sw.longseg, sw.nlong);
  launch_long_segsort(m, sw, st);
  (void)keep;
}

void build_csc_from_csr(const int* indptr, const int* indices, const double* data, int m, int n,
                        int nnz, const SparseWS& sw, cudaStream_t st) {
  const int cb = std::max(1, std::min((nnz + 255) / 256, 1184));
  k_csc_count<<<cb, 256, 0, st>>>(indptr, indices, m, sw.colcnt);
  k_scan<<<1, 1024, 0, st>>>(sw.colcnt, sw.colptr, n);
  const int pb = std::max(1, std::min((m + 255) / 256, 1184));
  k_csc_place<<<pb, 256, 0, st>>>(indptr, indices, data, m, sw.colptr, sw.colcnt, sw.trow,
                                  sw.tval);
  const int sb = std::max(1, std::min((n + 7) / 8, 2368));
  cudaMemsetAsync(sw.nlong, 0, sizeof(int), st);
  k_csc_segsort<<<sb, 256, 0, st>>>(sw.colptr, m, n, sw.colcnt, sw.trow, sw.tval, sw.rowidx,
                                    sw.cdata, sw.longseg, sw.nlong);
  launch_long_segsort(m, sw, st);
}

// ------------------------------------------------------------------------- //
// CG arguments (shared by the cluster and the cooperative kernels)
// ------------------------------------------------------------------------- //
struct CGArgs {
  int m, n; double inv_eta;
  const double* r; const double* c;
  const int* indptr; const int* indices; const double* data;
  const int* colptr; const int* rowidx; const double* cdata;
  const double* rhs; double* x;
  double* res; double* p; double* q;
  double* part;     // 3 * gridDim partials (cooperative kernel)
  double* dinv;     // D^-1 (cluster kernel)
  double rtol; int max_iter;
  double* info;     // {iterations, relative residual}
};

__device__ __forceinline__ double cg_block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // thread 0
}

// ------------------------------------------------------------------------- //
// Cooperative fallback (systems too large for one cluster's shared memory):
// grid-wide barriers; scalars from per-block partials summed in block order.
// ------------------------------------------------------------------------- //
__device__ __forceinline__ double cg_apply(const CGArgs& a, const double* v, int t) {
  if (t < a.m) {
    double acc = a.r[t] * v[t];
    for (int e = a.indptr[t]; e < a.indptr[t + 1]; ++e) acc += a.data[e] * v[a.m + a.indices[e]];
    return acc * a.inv_eta;
  }
  int j = t - a.m;
  double acc = a.c[j] * v[t];
  for (int e = a.colptr[j]; e < a.colptr[j + 1]; ++e) acc += a.cdata[e] * v[a.rowidx[e]];
  return acc * a.inv_eta;
}

__global__ void __launch_bounds__(256) k_pcg(CGArgs a) {
  // partial slots: [0, G) <p, Mp>, [G, 2G) <res, res>, [2G, 3G) <res, D^-1 res>;
  // a slot is rewritten only after a barrier every reader of it has passed.
  cg::grid_group grid = cg::this_grid();
  __shared__ double sh[32];
  __shared__ double bc[4];
  const int N = a.m + a.n;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthr = gridDim.x * blockDim.x;
  const int G = gridDim.x;
  double l_rz = 0.0, l_bb = 0.0;
  for (int t = tid; t < N; t += nthr) {
    double rv = a.rhs[t];
    double dg = (t < a.m) ? a.r[t] : a.c[t - a.m];
    double di = 1.0 / (dg * a.inv_eta);
    a.x[t] = 0.0; a.res[t] = rv; a.dinv[t] = di;
    double z = di * rv;
    a.p[t] = z;
    l_rz += rv * z; l_bb += rv * rv;
  }
  double b0 = cg_block_sum(l_rz, sh);
  __syncthreads();
  double b1 = cg_block_sum(l_bb, sh);
  if (threadIdx.x == 0) { a.part[2 * G + blockIdx.x] = b0; a.part[G + blockIdx.x] = b1; }
  grid.sync();
  double rz = 0.0, bnorm = 0.0;
  if (threadIdx.x == 0) {
    for (int k = 0; k < G; ++k) { rz += a.part[2 * G + k]; bnorm += a.part[G + k]; }
    bnorm = sqrt(bnorm);
    bc[2] = (bnorm > 0.0) ? 0.0 : 1.0;
  }
  __syncthreads();
  int it = 0;
  double rel = (bc[2] == 0.0) ? 1.0 : 0.0;
  if (bc[2] == 0.0) {
    while (it < a.max_iter) {
      double l_pq = 0.0;
      for (int t = tid; t < N; t += nthr) {
        double qv = cg_apply(a, a.p, t);
        a.q[t] = qv;
        l_pq += a.p[t] * qv;
      }
      double bp = cg_block_sum(l_pq, sh);
      if (threadIdx.x == 0) a.part[blockIdx.x] = bp;
      grid.sync();
      if (threadIdx.x == 0) {
        double pq = 0.0;
        for (int k = 0; k < G; ++k) pq += a.part[k];
        bc[0] = rz / pq;
      }
      __syncthreads();
      const double alpha = bc[0];
      double l_rr = 0.0, l_rz2 = 0.0;
      for (int t = tid; t < N; t += nthr) {
        a.x[t] += alpha * a.p[t];
        double rv = a.res[t] - alpha * a.q[t];
        a.res[t] = rv;
        l_rr += rv * rv;
        l_rz2 += rv * (a.dinv[t] * rv);
      }
      double c0 = cg_block_sum(l_rr, sh);
      __syncthreads();
      double c1 = cg_block_sum(l_rz2, sh);
      if (threadIdx.x == 0) { a.part[G + blockIdx.x] = c0; a.part[2 * G + blockIdx.x] = c1; }
      grid.sync();
      ++it;
      if (threadIdx.x == 0) {
        double rr = 0.0, rz2 = 0.0;
        for (int k = 0; k < G; ++k) { rr += a.part[G + k]; rz2 += a.part[2 * G + k]; }
        rel = sqrt(rr) / bnorm;
        bc[1] = rz2 / rz;
        rz = rz2;
        bc[2] = (rel > a.rtol) ? 0.0 : 1.0;
        bc[3] = rel;
      }
      __syncthreads();
      if (bc[2] != 0.0) break;
      const double beta = bc[1];
      for (int t = tid; t < N; t += nthr) a.p[t] = a.dinv[t] * a.res[t] + beta * a.p[t];
      grid.sync();
    }
    rel = bc[3];
  }
  if (tid == 0) { a.info[0] = (double)it; a.info[1] = rel; }
}

int cg_blocks(int N, int sms) {
  int b = (N + 255) / 256;
  int cap = sms < 64 ? sms : 64;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return b;
}

cudaError_t launch_pcg(int m, int n, double eta, const double* r, const double* c,
                       const int* indptr, const int* indices, const double* data,
                       const int* colptr, const int* rowidx, const double* cdata,
                       const double* rhs, double* x, double* res, double* p, double* q,
                       double* part, double rtol, int max_iter, double* info, int* flag,
                       int sms, cudaStream_t st) {
  CGArgs a;
  a.m = m; a.n = n; a.inv_eta = 1.0 / eta;
  a.r = r; a.c = c; a.indptr = indptr; a.indices = indices; a.data = data;
  a.colptr = colptr; a.rowidx = rowidx; a.cdata = cdata;
  a.rhs = rhs; a.x = x; a.res = res; a.p = p; a.q = q; a.part = part;
  a.rtol = rtol; a.max_iter = max_iter; a.info = info;
  bool used = false;
  cudaError_t ce = launch_pcg_cluster(m, n, eta, r, c, indptr, indices, data, colptr, rowidx,
                                      cdata, rhs, x, rtol, max_iter, info,
                                      flag, st, &used);
  if (used) return ce;
  const int N = m + n;
  a.dinv = q + N;   // (the cooperative path uses p globally; D^-1 goes after q)
  int blocks = cg_blocks(m + n, sms);
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((void*)k_pcg, dim3(blocks), dim3(256), args, 0, st);
}

// ------------------------------------------------------------------------- //
// Vector kernels (FP64, O(m + n))
// ------------------------------------------------------------------------- //
// A_i = F_i/eta - s, B_j = G_j/eta (FP64 and double-float copies)
__global__ void k_prep(const double* F, const double* G, int m, int n, double inv_eta,
                       double s, double* A64, double* B64, float2* Add, float2* Bdd) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m + n; t += gridDim.x * blockDim.x) {
    double v = (t < m) ? F[t] * inv_eta - s : G[t - m] * inv_eta;
    float hi = __double2float_rn(v);
    float lo = __double2float_rn(v - (double)hi);
    if (t < m) { if (A64) A64[t] = v; if (Add) Add[t] = make_float2(hi, lo); }
    else { if (B64) B64[t - m] = v; if (Bdd) Bdd[t - m] = make_float2(hi, lo); }
  }
}
void launch_prep(const double* F, const double* G, int m, int n, double eta, double s,
                 double* A64, double* B64, float2* Add, float2* Bdd, cudaStream_t st) {
  int N = m + n; int blocks = (N + 255) / 256; if (blocks > 512) blocks = 512;
  k_prep<<<blocks, 256, 0, st>>>(F, G, m, n, 1.0 / eta, s, A64, B64, Add, Bdd);
}

// trial increments Pt_i = alpha df_i / eta, Qt_j = alpha dg_j / eta
__global__ void k_trial_prep(const double* d, int m, int n, double scale, double* P64,
                             double* Q64, float2* Pdd, float2* Qdd) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m + n; t += gridDim.x * blockDim.x) {
    double v = d[t] * scale;
    float hi = __double2float_rn(v);
    float lo = __double2float_rn(v - (double)hi);
    if (t < m) { if (P64) P64[t] = v; if (Pdd) Pdd[t] = make_float2(hi, lo); }
    else { if (Q64) Q64[t - m] = v; if (Qdd) Qdd[t - m] = make_float2(hi, lo); }
  }
}
void launch_trial_prep(const double* d, int m, int n, double scale, double* P64, double* Q64,
                       float2* Pdd, float2* Qdd, cudaStream_t st) {
  int N = m + n; int blocks = (N + 255) / 256; if (blocks > 512) blocks = 512;
  k_trial_prep<<<blocks, 256, 0, st>>>(d, m, n, scale, P64, Q64, Pdd, Qdd);
}

// rhs = (a - r, b - c)
__global__ void k_grad(const double* a, const double* b, const double* r, const double* c,
                       int m, int n, double* g) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m + n; t += gridDim.x * blockDim.x)
    g[t] = (t < m) ? a[t] - r[t] : b[t - m] - c[t - m];
}
void launch_grad(const double* a, const double* b, const double* r, const double* c, int m,
                 int n, double* g, cudaStream_t st) {
  int N = m + n; int blocks = (N + 255) / 256; if (blocks > 512) blocks = 512;
  k_grad<<<blocks, 256, 0, st>>>(a, b, r, c, m, n, g);
}

// (log a; log b), once per bound problem
__global__ void k_log_ab(const double* a, const double* b, int m, int n, double* out) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m + n; t += gridDim.x * blockDim.x)
    out[t] = log((t < m) ? a[t] : b[t - m]);
}
void launch_log_ab(const double* a, const double* b, int m, int n, double* out, cudaStream_t st) {
  int N = m + n; int blocks = (N + 255) / 256; if (blocks > 512) blocks = 512;
  k_log_ab<<<blocks, 256, 0, st>>>(a, b, m, n, out);
}

// (F, G) += alpha d
// (F; G) += alpha d, then A = F/eta - s, B = G/eta (as k_prep) in the same launch
__global__ void k_axpy_prep(double* F, double* G, const double* d, int m, int n, double alpha,
                            double inv_eta, double s, double* A64, double* B64, float2* Add,
                            float2* Bdd) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m + n; t += gridDim.x * blockDim.x) {
    double v;
    if (t < m) { v = F[t] + alpha * d[t]; F[t] = v; v = v * inv_eta - s; }
    else { v = G[t - m] + alpha * d[t]; G[t - m] = v; v = v * inv_eta; }
    float hi = __double2float_rn(v);
    float lo = __double2float_rn(v - (double)hi);
    if (t < m) { if (A64) A64[t] = v; if (Add) Add[t] = make_float2(hi, lo); }
    else { if (B64) B64[t - m] = v; if (Bdd) Bdd[t - m] = make_float2(hi, lo); }
  }
}
void launch_axpy_prep(double* F, double* G, const double* d, int m, int n, double alpha,
                      double eta, double s, double* A64, double* B64, float2* Add, float2* Bdd,
                      cudaStream_t st) {
  int N = m + n; int blocks = (N + 255) / 256; if (blocks > 512) blocks = 512;
  k_axpy_prep<<<blocks, 256, 0, st>>>(F, G, d, m, n, alpha, 1.0 / eta, s, A64, B64, Add, Bdd);
}

// outer update (reading R2): f = F - Phi; Phi = F; F = F + f (same for G)
__global__ void k_outer(double* F, double* G, double* Phi, double* Psi, int m, int n) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m + n; t += gridDim.x * blockDim.x) {
    double* X = (t < m) ? F : G;
    double* Y = (t < m) ? Phi : Psi;
    int k = (t < m) ? t : t - m;
    double v = X[k];
    double f = v - Y[k];
    Y[k] = v;
    X[k] = v + f;
  }
}
void launch_outer(double* F, double* G, double* Phi, double* Psi, int m, int n, cudaStream_t st) {
  int N = m + n; int blocks = (N + 255) / 256; if (blocks > 512) blocks = 512;
  k_outer<<<blocks, 256, 0, st>>>(F, G, Phi, Psi, m, n);
}

// deterministic dot products: out[0] = <x1, y1>, out[1] = <x2, y2>
__global__ void __launch_bounds__(256) k_dot2(const double* x1, const double* y1,
                                              const double* x2, const double* y2, int N,
                                              double* out) {
  __shared__ double sh[32];
  double s1 = 0.0, s2 = 0.0;
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    s1 += x1[t] * y1[t];
    if (x2) s2 += x2[t] * y2[t];
  }
  double b1 = cg_block_sum(s1, sh);
  __syncthreads();
  double b2 = cg_block_sum(s2, sh);
  if (threadIdx.x == 0) { out[0] = b1; out[1] = b2; }
}
void launch_dot2(const double* x1, const double* y1, const double* x2, const double* y2, int N,
                 double* out, cudaStream_t st) {
  k_dot2<<<1, 256, 0, st>>>(x1, y1, x2, y2, N, out);
}

// certificate helpers --------------------------------------------------------
// xs_i = min(a_i / r_i, 1); u_i = F_i / s - eta
__global__ void k_cert_pre(const double* a, const double* r, const double* F, int m, double s,
                           double eta, double* xs, double* u) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    double q = a[i] / r[i];
    xs[i] = q < 1.0 ? q : 1.0;
    u[i] = F[i] / s - eta;
  }
}
// ys_j = min(b_j / c1_j, 1); ec_j = b_j - ys_j c1_j
__global__ void k_cert_mid(const double* b, const double* c1, int n, double* ys, double* ec) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double q = b[j] / c1[j];
    double y = q < 1.0 ? q : 1.0;
    ys[j] = y;
    ec[j] = b[j] - y * c1[j];
  }
}
// final scalars: cost, UB, LB, gap (one CTA, fixed order).  LB is the larger of
// the two c-transform bounds: <a, u2> + <b, v> (entropic dual) and
// <a, u2T> + <b, vT> (support-tree dual).
__global__ void __launch_bounds__(256) k_cert_final(const double* a, const double* b,
                                                    const double* rr, const double* cr,
                                                    const double* cp, const double* tc,
                                                    const double* u2, const double* v,
                                                    const double* u2T, const double* vT,
                                                    int m, int n, double* out4, double* lb2) {
  __shared__ double sh[32];
  double s_cost = 0, s_cr = 0, s_er = 0, s_ert = 0, s_lb = 0, s_lbt = 0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double er = a[i] - rr[i];
    s_cost += cp[i]; s_cr += cr[i]; s_er += fabs(er); s_ert += er * tc[i];
    s_lb += a[i] * u2[i];
    s_lbt += a[i] * u2T[i];
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) { s_lb += b[j] * v[j]; s_lbt += b[j] * vT[j]; }
  double t0 = cg_block_sum(s_cost, sh); __syncthreads();
  double t1 = cg_block_sum(s_cr, sh); __syncthreads();
  double t2 = cg_block_sum(s_er, sh); __syncthreads();
  double t3 = cg_block_sum(s_ert, sh); __syncthreads();
  double t4 = cg_block_sum(s_lb, sh); __syncthreads();
  double t5 = cg_block_sum(s_lbt, sh);
  if (threadIdx.x == 0) {
    double ub = t1 + (t2 > 0.0 ? t3 / t2 : 0.0);
    double lb = fmax(t4, t5);
    double gap = (lb > 0.0) ? (ub - lb) / lb : (ub - lb) / fmax(fabs(ub), 1e-300);
    out4[0] = t0; out4[1] = ub; out4[2] = lb; out4[3] = gap;
    if (lb2) { lb2[0] = t4; lb2[1] = t5; }
  }
}
void launch_cert_pre(const double* a, const double* r, const double* F, int m, double s,
                     double eta, double* xs, double* u, cudaStream_t st) {
  k_cert_pre<<<(m + 255) / 256, 256, 0, st>>>(a, r, F, m, s, eta, xs, u);
}
void launch_cert_mid(const double* b, const double* c1, int n, double* ys, double* ec,
                     cudaStream_t st) {
  k_cert_mid<<<(n + 255) / 256, 256, 0, st>>>(b, c1, n, ys, ec);
}
void launch_cert_final(const double* a, const double* b, const double* rr, const double* cr,
                       const double* cp, const double* tc, const double* u2, const double* v,
                       const double* u2T, const double* vT, int m, int n, double* out4,
                       double* lb2, cudaStream_t st) {
  k_cert_final<<<1, 256, 0, st>>>(a, b, rr, cr, cp, tc, u2, v, u2T, vT, m, n, out4, lb2);
}

// cast helpers
__global__ void k_d2f(const double* x, float* y, size_t N) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < N;
       t += (size_t)gridDim.x * blockDim.x)
    y[t] = __double2float_rn(x[t]);
}
__global__ void k_f2d(const float* x, double* y, size_t N) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < N;
       t += (size_t)gridDim.x * blockDim.x)
    y[t] = (double)x[t];
}
void launch_d2f(const double* x, float* y, size_t N, cudaStream_t st) {
  k_d2f<<<1024, 256, 0, st>>>(x, y, N);
}
void launch_f2d(const float* x, double* y, size_t N, cudaStream_t st) {
  k_f2d<<<1024, 256, 0, st>>>(x, y, N);
}

}  // namespace pins
