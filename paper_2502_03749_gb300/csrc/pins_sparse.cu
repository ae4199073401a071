// Sparse side of the Newton step (Algorithm 2): CSC assembly of the kept
// coupling entries, the truncated Jacobi-preconditioned CG on
//   M d = rhs,   M = (1/eta) [[diag r, S], [S^T, diag c]],
// and the O(m + n) vector kernels of the solver (FP64).
//
// FP64 on GB300 runs at ~1/64 of the FP32 rate (~19 SM-cycles per warp-wide FP64
// instruction), so scalar bookkeeping is done by one thread and broadcast, and the
// vector work is spread over a thread-block cluster.
#include <cooperative_groups.h>
#include "pins_kernels.h"

namespace cg = cooperative_groups;

namespace pins {

// exclusive scan of cnt[0..len) into ptr[0..len], resets cnt to 0
__global__ void __launch_bounds__(1024) k_scan(int* cnt, int* ptr, int len) {
  __shared__ int sh[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < len; base += 1024) {
    int t = base + threadIdx.x;
    int v = (t < len) ? cnt[t] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int add = (threadIdx.x >= o) ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += add;
      __syncthreads();
    }
    if (t < len) { ptr[t] = carry + sh[threadIdx.x] - v; cnt[t] = 0; }
    __syncthreads();
    if (threadIdx.x == 0) carry += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) ptr[len] = carry;
}
void launch_scan(int* cnt, int* ptr, int len, cudaStream_t st) {
  k_scan<<<1, 1024, 0, st>>>(cnt, ptr, len);
}

// ------------------------------------------------------------------------- //
// CSC from the row-ordered CSR.  Up to PINS_CSC_SMEM entries: one CTA sorts the
// keys (j << 32 | i) by a bitonic network in shared memory (payload: CSR
// position) and derives colptr from the sorted columns.  Larger: a stable
// counting sort over row chunks.  Either way the rows of a column come out
// ascending, independent of timing.
// ------------------------------------------------------------------------- //
#define PINS_CSC_SMEM 16384

__global__ void __launch_bounds__(1024)
k_csc_sort(const int* indptr, const int* indices, const double* data, int m, int n,
           int* colptr, int* rowidx, double* cdata) {
  extern __shared__ unsigned char csc_smem[];
  const int K = indptr[m];
  unsigned int P2 = 1;
  while (P2 < (unsigned int)K) P2 <<= 1;
  unsigned long long* key = reinterpret_cast<unsigned long long*>(csc_smem);
  int* pos = reinterpret_cast<int*>(key + P2);
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    for (int e = indptr[i]; e < indptr[i + 1]; ++e) {
      key[e] = ((unsigned long long)(unsigned int)indices[e] << 32) | (unsigned int)i;
      pos[e] = e;
    }
  for (unsigned int q = K + threadIdx.x; q < P2; q += blockDim.x) { key[q] = ~0ull; pos[q] = -1; }
  __syncthreads();
  for (unsigned int k = 2; k <= P2; k <<= 1) {
    for (unsigned int jv = k >> 1; jv > 0; jv >>= 1) {
      for (unsigned int t = threadIdx.x; t < P2; t += blockDim.x) {
        unsigned int l = t ^ jv;
        if (l > t) {
          bool up = ((t & k) == 0);
          unsigned long long ka = key[t], kb = key[l];
          if (up ? (ka > kb) : (ka < kb)) {
            key[t] = kb; key[l] = ka;
            int pa = pos[t]; pos[t] = pos[l]; pos[l] = pa;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int q = threadIdx.x; q < K; q += blockDim.x) {
    const int j = (int)(key[q] >> 32);
    rowidx[q] = (int)(key[q] & 0xffffffffu);
    cdata[q] = data[pos[q]];
    const int jprev = (q == 0) ? -1 : (int)(key[q - 1] >> 32);
    for (int c = jprev + 1; c <= j; ++c) colptr[c] = q;      // columns starting here
    if (q == K - 1) for (int c = j + 1; c <= n; ++c) colptr[c] = K;
  }
  if (K == 0) for (int c = threadIdx.x; c <= n; c += blockDim.x) colptr[c] = 0;
}

__device__ __forceinline__ void chunk_rows(int c, int chunks, int m, int& r0, int& r1) {
  const int R = (m + chunks - 1) / chunks;
  r0 = min(m, c * R);
  r1 = min(m, r0 + R);
}
__global__ void k_csc_count(const int* indptr, const int* indices, int m, int n, int chunks,
                            int* cnt) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < chunks; c += gridDim.x * blockDim.x) {
    int r0, r1; chunk_rows(c, chunks, m, r0, r1);
    for (int e = indptr[r0]; e < indptr[r1]; ++e) cnt[(size_t)c * n + indices[e]] += 1;
  }
}
__global__ void k_csc_colscan(int* cnt, int chunks, int n, int* coltot) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    int run = 0;
    for (int c = 0; c < chunks; ++c) {
      int v = cnt[(size_t)c * n + j];
      cnt[(size_t)c * n + j] = run;
      run += v;
    }
    coltot[j] = run;
  }
}
__global__ void k_csc_scatter(const int* indptr, const int* indices, const double* data, int m,
                              int n, int chunks, int* off, const int* colptr, int* rowidx,
                              double* cdata) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < chunks; c += gridDim.x * blockDim.x) {
    int r0, r1; chunk_rows(c, chunks, m, r0, r1);
    for (int i = r0; i < r1; ++i)
      for (int e = indptr[i]; e < indptr[i + 1]; ++e) {
        const int j = indices[e];
        const int pos = colptr[j] + off[(size_t)c * n + j]++;
        rowidx[pos] = i;
        cdata[pos] = data[e];
      }
  }
}

void build_csc_from_csr(const int* indptr, const int* indices, const double* data, int m, int n,
                        int nnz, const SparseWS& sw, cudaStream_t st) {
  if (nnz <= PINS_CSC_SMEM) {
    unsigned int P2 = 1;
    while (P2 < (unsigned int)nnz) P2 <<= 1;
    const size_t smem = (size_t)P2 * (sizeof(unsigned long long) + sizeof(int));
    static bool configured = false;
    if (!configured) {
      cudaFuncSetAttribute(k_csc_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)((size_t)PINS_CSC_SMEM * 12));
      configured = true;
    }
    k_csc_sort<<<1, 1024, smem, st>>>(indptr, indices, data, m, n, sw.colptr, sw.rowidx, sw.cdata);
    return;
  }
  const int chunks = m < PINS_CSC_CHUNKS ? m : PINS_CSC_CHUNKS;
  cudaMemsetAsync(sw.chunkcnt, 0, sizeof(int) * (size_t)chunks * n, st);
  k_csc_count<<<(chunks + 255) / 256, 256, 0, st>>>(indptr, indices, m, n, chunks, sw.chunkcnt);
  k_csc_colscan<<<(n + 255) / 256, 256, 0, st>>>(sw.chunkcnt, chunks, n, sw.colcnt);
  k_scan<<<1, 1024, 0, st>>>(sw.colcnt, sw.colptr, n);
  k_csc_scatter<<<(chunks + 255) / 256, 256, 0, st>>>(indptr, indices, data, m, n, chunks,
                                                      sw.chunkcnt, sw.colptr, sw.rowidx, sw.cdata);
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
                       double* part, double rtol, int max_iter, double* info, int sms,
                       cudaStream_t st) {
  CGArgs a;
  a.m = m; a.n = n; a.inv_eta = 1.0 / eta;
  a.r = r; a.c = c; a.indptr = indptr; a.indices = indices; a.data = data;
  a.colptr = colptr; a.rowidx = rowidx; a.cdata = cdata;
  a.rhs = rhs; a.x = x; a.res = res; a.p = p; a.q = q; a.part = part;
  a.rtol = rtol; a.max_iter = max_iter; a.info = info;
  bool used = false;
  cudaError_t ce = launch_pcg_cluster(m, n, eta, r, c, indptr, indices, data, colptr, rowidx,
                                      cdata, rhs, x, rtol, max_iter, info,
                                      reinterpret_cast<int*>(part + 3 * 64), st, &used);
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

// (F, G) += alpha d
__global__ void k_axpy2(double* F, double* G, const double* d, int m, int n, double alpha) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m + n; t += gridDim.x * blockDim.x) {
    if (t < m) F[t] += alpha * d[t]; else G[t - m] += alpha * d[t];
  }
}
void launch_axpy2(double* F, double* G, const double* d, int m, int n, double alpha,
                  cudaStream_t st) {
  int N = m + n; int blocks = (N + 255) / 256; if (blocks > 512) blocks = 512;
  k_axpy2<<<blocks, 256, 0, st>>>(F, G, d, m, n, alpha);
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
// final scalars: cost, UB, LB, gap (one CTA, fixed order)
__global__ void __launch_bounds__(256) k_cert_final(const double* a, const double* b,
                                                    const double* rr, const double* cr,
                                                    const double* cp, const double* tc,
                                                    const double* u2, const double* v,
                                                    int m, int n, double* out4) {
  __shared__ double sh[32];
  double s_cost = 0, s_cr = 0, s_er = 0, s_ert = 0, s_lb = 0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double er = a[i] - rr[i];
    s_cost += cp[i]; s_cr += cr[i]; s_er += fabs(er); s_ert += er * tc[i];
    s_lb += a[i] * u2[i];
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) s_lb += b[j] * v[j];
  double t0 = cg_block_sum(s_cost, sh); __syncthreads();
  double t1 = cg_block_sum(s_cr, sh); __syncthreads();
  double t2 = cg_block_sum(s_er, sh); __syncthreads();
  double t3 = cg_block_sum(s_ert, sh); __syncthreads();
  double t4 = cg_block_sum(s_lb, sh);
  if (threadIdx.x == 0) {
    double ub = t1 + (t2 > 0.0 ? t3 / t2 : 0.0);
    double lb = t4;
    double gap = (lb > 0.0) ? (ub - lb) / lb : (ub - lb) / fmax(fabs(ub), 1e-300);
    out4[0] = t0; out4[1] = ub; out4[2] = lb; out4[3] = gap;
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
                       int m, int n, double* out4, cudaStream_t st) {
  k_cert_final<<<1, 256, 0, st>>>(a, b, rr, cr, cp, tc, u2, v, m, n, out4);
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
