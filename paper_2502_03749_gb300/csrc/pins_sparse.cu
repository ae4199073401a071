// Sparse side of the Newton step (Algorithm 2): CSR/CSC assembly of the kept
// coupling entries, the truncated Jacobi-preconditioned CG on
//   M d = rhs,   M = (1/eta) [[diag r, S], [S^T, diag c]],
// and the O(m + n) vector kernels of the solver (FP64).
#include <cooperative_groups.h>
#include "pins_kernels.h"

namespace cg = cooperative_groups;

namespace pins {

// ------------------------------------------------------------------------- //
// CSR / CSC assembly from the COO list of kept entries (linear index + key).
// Positions inside a row (column) come from atomics, then each row (column) is
// sorted by column (row) index, so the final arrays do not depend on timing.
// ------------------------------------------------------------------------- //
__global__ void k_coo_count(const long long* idx, int nnz, int n, int* rowcnt, int* colcnt) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += gridDim.x * blockDim.x) {
    long long l = idx[e];
    int i = (int)(l / n), j = (int)(l - (long long)i * n);
    atomicAdd(rowcnt + i, 1);
    atomicAdd(colcnt + j, 1);
  }
}

// exclusive scan of cnt[0..len) into ptr[0..len], resets cnt to 0 (cursor)
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

// value of a kept entry: X~_ij = exp(key / eta) (FP64 key) or exp(z) (mixed key = z)
__global__ void k_coo_scatter(const long long* idx, const double* key, int nnz, int n,
                              double key_scale, const int* rowptr, int* rowcur,
                              int* csr_col, double* csr_val, const int* colptr, int* colcur,
                              int* csc_row, double* csc_val) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += gridDim.x * blockDim.x) {
    long long l = idx[e];
    int i = (int)(l / n), j = (int)(l - (long long)i * n);
    double val = exp(key[e] * key_scale);
    int pr = rowptr[i] + atomicAdd(rowcur + i, 1);
    csr_col[pr] = j; csr_val[pr] = val;
    int pc = colptr[j] + atomicAdd(colcur + j, 1);
    csc_row[pc] = i; csc_val[pc] = val;
  }
}

// insertion sort of each segment by index (segments are short: ~2 entries)
__global__ void k_segment_sort(const int* ptr, int len, int* ind, double* val) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < len; s += gridDim.x * blockDim.x) {
    int lo = ptr[s], hi = ptr[s + 1];
    for (int a = lo + 1; a < hi; ++a) {
      int ki = ind[a]; double kv = val[a];
      int b = a - 1;
      while (b >= lo && ind[b] > ki) { ind[b + 1] = ind[b]; val[b + 1] = val[b]; --b; }
      ind[b + 1] = ki; val[b + 1] = kv;
    }
  }
}

void build_csr(const long long* coo_idx, const double* coo_key, int nnz, int m, int n,
               double key_scale, const SparseWS& sw, cudaStream_t st) {
  cudaMemsetAsync(sw.rowcnt, 0, sizeof(int) * m, st);
  cudaMemsetAsync(sw.colcnt, 0, sizeof(int) * n, st);
  int blocks = (nnz + 255) / 256; if (blocks < 1) blocks = 1; if (blocks > 1024) blocks = 1024;
  k_coo_count<<<blocks, 256, 0, st>>>(coo_idx, nnz, n, sw.rowcnt, sw.colcnt);
  k_scan<<<1, 1024, 0, st>>>(sw.rowcnt, sw.indptr, m);
  k_scan<<<1, 1024, 0, st>>>(sw.colcnt, sw.colptr, n);
  k_coo_scatter<<<blocks, 256, 0, st>>>(coo_idx, coo_key, nnz, n, key_scale, sw.indptr,
                                        sw.rowcnt, sw.indices, sw.data, sw.colptr, sw.colcnt,
                                        sw.rowidx, sw.cdata);
  k_segment_sort<<<(m + 255) / 256, 256, 0, st>>>(sw.indptr, m, sw.indices, sw.data);
  k_segment_sort<<<(n + 255) / 256, 256, 0, st>>>(sw.colptr, n, sw.rowidx, sw.cdata);
}

// CSC from a given CSR (for the step-level CG entry point)
__global__ void k_csr_count_cols(const int* indptr, const int* indices, int m, int* colcnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    for (int e = indptr[i]; e < indptr[i + 1]; ++e) atomicAdd(colcnt + indices[e], 1);
}
__global__ void k_csr_scatter_cols(const int* indptr, const int* indices, const double* data,
                                   int m, const int* colptr, int* colcur, int* rowidx,
                                   double* cdata) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    for (int e = indptr[i]; e < indptr[i + 1]; ++e) {
      int j = indices[e];
      int pc = colptr[j] + atomicAdd(colcur + j, 1);
      rowidx[pc] = i; cdata[pc] = data[e];
    }
}
void build_csc_from_csr(const int* indptr, const int* indices, const double* data, int m,
                        int n, int* colcnt, int* colptr, int* rowidx, double* cdata,
                        cudaStream_t st) {
  cudaMemsetAsync(colcnt, 0, sizeof(int) * n, st);
  k_csr_count_cols<<<(m + 255) / 256, 256, 0, st>>>(indptr, indices, m, colcnt);
  k_scan<<<1, 1024, 0, st>>>(colcnt, colptr, n);
  k_csr_scatter_cols<<<(m + 255) / 256, 256, 0, st>>>(indptr, indices, data, m, colptr, colcnt,
                                                      rowidx, cdata);
  k_segment_sort<<<(n + 255) / 256, 256, 0, st>>>(colptr, n, rowidx, cdata);
}

// ------------------------------------------------------------------------- //
// Truncated PCG (Jacobi), cooperative: a few CTAs, grid-wide barriers.
// Reduction order is fixed (per-thread strided sums, block tree, partials summed
// in block order by every CTA), so every CTA sees identical scalars.
// ------------------------------------------------------------------------- //
struct CGArgs {
  int m, n; double inv_eta;
  const double* r; const double* c;
  const int* indptr; const int* indices; const double* data;
  const int* colptr; const int* rowidx; const double* cdata;
  const double* rhs; double* x;
  double* res; double* p; double* q;
  double* part;     // 3 * gridDim partials (see k_pcg)
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

__device__ __forceinline__ double cg_apply(const CGArgs& a, const double* v, int t) {
  // (M v)_t
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
__device__ __forceinline__ double cg_dinv(const CGArgs& a, int t) {
  double d = (t < a.m) ? a.r[t] : a.c[t - a.m];
  return 1.0 / (d * a.inv_eta);
}

__global__ void __launch_bounds__(256) k_pcg(CGArgs a) {
  // partial slots: [0, G) <p, Mp>, [G, 2G) <res, res>, [2G, 3G) <res, D^-1 res>.
  // A slot is rewritten only after a barrier that every reader of its previous
  // contents has passed.
  cg::grid_group grid = cg::this_grid();
  __shared__ double sh[32];
  const int N = a.m + a.n;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthr = gridDim.x * blockDim.x;
  const int G = gridDim.x;
  double l_rz = 0.0, l_bb = 0.0;
  for (int t = tid; t < N; t += nthr) {
    double rv = a.rhs[t];
    a.x[t] = 0.0; a.res[t] = rv;
    double z = cg_dinv(a, t) * rv;
    a.p[t] = z;
    l_rz += rv * z; l_bb += rv * rv;
  }
  double b0 = cg_block_sum(l_rz, sh);
  double b1 = cg_block_sum(l_bb, sh);
  if (threadIdx.x == 0) { a.part[2 * G + blockIdx.x] = b0; a.part[G + blockIdx.x] = b1; }
  grid.sync();
  double rz = 0.0, bb = 0.0;
  for (int k = 0; k < G; ++k) { rz += a.part[2 * G + k]; bb += a.part[G + k]; }
  const double bnorm = sqrt(bb);
  int it = 0;
  double rel = (bnorm > 0.0) ? 1.0 : 0.0;
  if (bnorm > 0.0) {
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
      double pq = 0.0;
      for (int k = 0; k < G; ++k) pq += a.part[k];
      double alpha = rz / pq;
      double l_rr = 0.0, l_rz2 = 0.0;
      for (int t = tid; t < N; t += nthr) {
        a.x[t] += alpha * a.p[t];
        double rv = a.res[t] - alpha * a.q[t];
        a.res[t] = rv;
        l_rr += rv * rv;
        l_rz2 += rv * (cg_dinv(a, t) * rv);
      }
      double c0 = cg_block_sum(l_rr, sh);
      double c1 = cg_block_sum(l_rz2, sh);
      if (threadIdx.x == 0) { a.part[G + blockIdx.x] = c0; a.part[2 * G + blockIdx.x] = c1; }
      grid.sync();
      double rr = 0.0, rz2 = 0.0;
      for (int k = 0; k < G; ++k) { rr += a.part[G + k]; rz2 += a.part[2 * G + k]; }
      ++it;
      rel = sqrt(rr) / bnorm;
      if (!(rel > a.rtol)) break;   // also stops on NaN
      double beta = rz2 / rz;
      rz = rz2;
      for (int t = tid; t < N; t += nthr) a.p[t] = cg_dinv(a, t) * a.res[t] + beta * a.p[t];
      grid.sync();
    }
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

// y[0..N) += alpha x  (F,G stacked as separate arrays)
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

// deterministic dot products: out[0] = <x, y> (+ optional second pair)
__global__ void __launch_bounds__(1024) k_dot2(const double* x1, const double* y1,
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
  k_dot2<<<1, 1024, 0, st>>>(x1, y1, x2, y2, N, out);
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
__global__ void __launch_bounds__(1024) k_cert_final(const double* a, const double* b,
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
  k_cert_final<<<1, 1024, 0, st>>>(a, b, rr, cr, cp, tc, u2, v, m, n, out4);
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
