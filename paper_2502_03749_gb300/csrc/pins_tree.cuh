// Support-tree dual of the certificate's lower bound (reading R9 (ii)).
//
// Input: the `ne` largest plan entries as a CSR pattern (row-major order, so
// edge index e orders ties by linear index i*n+j).  Nodes are the rows 0..m-1
// and the columns m..m+n-1.  The kernel
//   1. ranks the edges by the FP64 key k_ij = (F_i + G_j) - s (C_ij + eta)
//      (descending, ties to the lower edge index): a strict total order;
//   2. builds the maximum-weight spanning forest under that order by Boruvka's
//      algorithm (every component hooks along its best incident edge; with a
//      strict order the chosen edges form a forest apart from mutual pairs, and
//      the forest equals Kruskal's);
//   3. roots each tree at its lowest node, which keeps its entropic potential
//      (rows F_i/s - eta, columns G_j/s), and walks the tree level by level,
//      giving every other node the value that makes its tree edge tight,
//      u_i + v_j = C_ij.
// One CTA does all of it; phases are separated by __syncthreads and every loop
// ends when a phase changes nothing (each has a fixed cap as well).
#pragma once

namespace pins {

#define PINS_TREE_TPB 1024

struct TreeWS {
  int* erow;                   // ne: row of edge e
  unsigned long long* okey;    // ne: order-preserving image of k_e
  int* eflag;                  // ne: 1 if e is a forest edge
  int* comp;                   // V: component pointer (root: comp[v] == v)
  unsigned long long* bkey;    // V: best incident key of a component root
  int* be;                     // V: best incident edge of a component root
  int* lvl;                    // V: depth below the tree's root, -1 unknown
  int* minid;                  // V: lowest node of a component
  double* pot;                 // V: potentials (rows, then columns)
};

__device__ __forceinline__ unsigned long long key_order64(double k) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(k);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

template <class P>
__device__ __forceinline__ double tree_cost(const PassArgs& p, int i, int j) {
  if constexpr (P::MIXED) return __dmul_rn(p.cscale, (double)P::cost(p, i, j));
  else return P::cost(p, i, j);
}

template <class P>
__global__ void __launch_bounds__(PINS_TREE_TPB)
k_tree_duals(PassArgs p, const int* __restrict__ indptr, const int* __restrict__ indices, int ne,
             TreeWS tw, double* __restrict__ uT, int* err) {
  const int m = p.m, n = p.n, V = m + n;
  const int t0 = threadIdx.x, T = blockDim.x;
  // ---- edges: row, order key; nodes: singleton components ----
  for (int i = t0; i < m; i += T)
    for (int e = indptr[i]; e < indptr[i + 1]; ++e) {
      const int j = indices[e];
      const double c = tree_cost<P>(p, i, j);
      const double k = __dsub_rn(__dadd_rn(p.F[i], p.G[j]), __dmul_rn(p.s, __dadd_rn(c, p.eta)));
      tw.erow[e] = i;
      tw.okey[e] = key_order64(k);
      tw.eflag[e] = 0;
    }
  for (int v = t0; v < V; v += T) { tw.comp[v] = v; tw.lvl[v] = -1; }
  __syncthreads();
  // ---- Boruvka rounds ----
  for (int round = 0; round < 64; ++round) {
    for (int v = t0; v < V; v += T) { tw.bkey[v] = 0ull; tw.be[v] = 0x7fffffff; }
    __syncthreads();
    for (int e = t0; e < ne; e += T) {
      const int ci = tw.comp[tw.erow[e]], cj = tw.comp[m + indices[e]];
      if (ci != cj) {
        atomicMax(tw.bkey + ci, tw.okey[e]);
        atomicMax(tw.bkey + cj, tw.okey[e]);
      }
    }
    __syncthreads();
    for (int e = t0; e < ne; e += T) {
      const int ci = tw.comp[tw.erow[e]], cj = tw.comp[m + indices[e]];
      if (ci != cj) {
        const unsigned long long k = tw.okey[e];
        if (k == tw.bkey[ci]) atomicMin(tw.be + ci, e);
        if (k == tw.bkey[cj]) atomicMin(tw.be + cj, e);
      }
    }
    __syncthreads();
    // hook: a root follows its best edge; of a mutual pair only the higher root
    // hooks.  The new parents are staged in lvl[] because comp[] is read here.
    int hooked = 0;
    for (int c = t0; c < V; c += T) {
      const int e = tw.be[c];
      if (tw.comp[c] != c || e == 0x7fffffff) continue;
      const int ci = tw.comp[tw.erow[e]], cj = tw.comp[m + indices[e]];
      const int other = (ci == c) ? cj : ci;
      tw.eflag[e] = 1;
      if (tw.be[other] == e && c < other) continue;
      tw.lvl[c] = other;
      hooked = 1;
    }
    if (!__syncthreads_or(hooked)) break;
    for (int c = t0; c < V; c += T)
      if (tw.lvl[c] >= 0) { tw.comp[c] = tw.lvl[c]; tw.lvl[c] = -1; }
    __syncthreads();
    // pointer jumping until every node points at its component's root
    for (int it = 0; it < 64; ++it) {
      int changed = 0;
      for (int v = t0; v < V; v += T) {
        const int a = tw.comp[v], b = tw.comp[a];
        if (a != b) { tw.comp[v] = b; changed = 1; }
      }
      if (!__syncthreads_or(changed)) break;
      if (it == 63 && t0 == 0 && err) atomicOr(err, 32);
    }
  }
  // ---- roots: the lowest node of each component keeps its entropic potential ----
  for (int v = t0; v < V; v += T) tw.minid[v] = 0x7fffffff;
  __syncthreads();
  for (int v = t0; v < V; v += T) atomicMin(tw.minid + tw.comp[v], v);
  __syncthreads();
  for (int v = t0; v < V; v += T)
    if (tw.minid[tw.comp[v]] == v) {
      tw.pot[v] = (v < m) ? __dsub_rn(__ddiv_rn(p.F[v], p.s), p.eta) : __ddiv_rn(p.G[v - m], p.s);
      tw.lvl[v] = 0;
    }
  __syncthreads();
  // ---- level-by-level walk along the forest edges ----
  for (int depth = 0; depth < V; ++depth) {
    int grew = 0;
    for (int e = t0; e < ne; e += T) {
      if (!tw.eflag[e]) continue;
      const int i = tw.erow[e], y = m + indices[e];
      const int li = tw.lvl[i], ly = tw.lvl[y];
      if (li == depth && ly < 0) {
        tw.pot[y] = __dsub_rn(tree_cost<P>(p, i, y - m), tw.pot[i]);
        tw.lvl[y] = depth + 1;
        grew = 1;
      } else if (ly == depth && li < 0) {
        tw.pot[i] = __dsub_rn(tree_cost<P>(p, i, y - m), tw.pot[y]);
        tw.lvl[i] = depth + 1;
        grew = 1;
      }
    }
    if (!__syncthreads_or(grew)) break;
  }
  for (int i = t0; i < m; i += T) uT[i] = tw.pot[i];
}

}  // namespace pins
