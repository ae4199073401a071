"""FP64 CPU oracle of PINS (Proximal Iterations with sparse Newton and Sinkhorn).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the timed CPU
baseline of the benchmark may import this module.  The CUDA library never calls it
and shares no code with it.

It is plain NumPy float64, written step by step in the order of Algorithm 2 of
the paper, with dense m x n matrices.  Every function names the passage it
restates.  It is slow on purpose: no blocking, no fusion, no reordering.

Notation.  Algorithm 2 shifts the cost by C^k = C - eta log X^k and solves the
entropic subproblem (Eq. eppa-sub) through the primal map of Eq. eppa_x,
    X~^k(f, g) = exp((f 1^T + 1 g^T - C^k - eta E) / eta).
With X^0 = E and X^{l+1} = X~^l(f^l, g^l), unrolling the recursion gives
    log X^k = (Phi 1^T + 1 Psi^T - k (C + eta E)) / eta,   Phi = sum_{l<k} f^l,
so with F = Phi + f, G = Psi + g and s = k + 1,
    log X~^k(f, g)_ij = (F_i + G_j - s (C_ij + eta)) / eta.            (*)
The oracle carries (Phi, Psi, F, G, s) and never stores X^k.  The test-suite pins
(*) against the literal recursion.

Readings where the paper is silent (each is also listed in the design notes):
  R1  X^0 = E (all ones), f^0 = g^0 = 0.
  R2  Warm start (Section 3.2, last paragraph): subproblem k+1 starts from the
      terminal duals (f^k, g^k) of subproblem k, i.e. F <- F + f^k, G <- G + g^k.
  R3  Sinkhorn block order is Gauss-Seidel (the g update uses the new f), Alg. 1.
  R4  T1, T2, K are caps (Alg. 2 inputs).  The warm-up also ends once the row
      residual measured in a row half-step is <= tol_marg (checked every
      `sinkhorn_check_every` iterations); Newton ends once the l1 marginal
      residual is <= tol_marg.
  R5  Sparsify keeps the K = round(gamma (m + n - 1)) largest entries of X~
      (ties -> lower row-major index); gamma = 1 gives the density
      (3n - 1)/(2n^2) of Theorem 2 for m = n.
  R6  CG is Jacobi-preconditioned, x0 = 0, stops at relative residual cg_rtol or
      max_cg iterations.
  R7  Armijo: alpha in {1, beta, beta^2, ...} (at most max_backtrack halvings) on
      P^k(x + alpha d) - P^k(x) >= c1 alpha grad^T d, where the left side is
      evaluated as alpha(<a,df> + <b,dg>) - eta sum X~ expm1(alpha (df_i + dg_j) / eta),
      the same quantity free of cancellation.  If no alpha passes, one Sinkhorn
      iteration is taken instead.
  R8  Residual = ||X~ 1 - a||_1 + ||X~^T 1 - b||_1.
  R9  Outer stop: certified relative gap (UB - LB) / LB <= tol_gap, or K.
      LB: the larger of two LP weak-duality bounds, each the double c-transform
      of a row potential: (i) u = F/s - eta, the subproblem's own dual, whose
      bound trails OPT by O(eta/s); (ii) the support-tree dual: potentials that
      satisfy u_i + v_j = C_ij exactly on a maximum-weight spanning forest of
      the 2(m + n - 1) largest plan entries (complementary slackness on the
      plan's support), which is an optimal LP dual once the plan has
      concentrated on an optimal basis.  UB: cost of the
      Altschuler-Weed-Rigollet rounding of X~ onto the transport polytope.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np


# --------------------------------------------------------------------------- #
# Configuration (defaults: Appendix E.1 hyperparameters)
# --------------------------------------------------------------------------- #
@dataclasses.dataclass
class Config:
    eta: float = 1e-2            # proximal / entropic parameter
    T1: int = 100                # Sinkhorn warm-up cap
    T2: int = 50                 # Newton cap
    K: int = 250                 # outer (EPPA) cap
    tol_marg: float = 1e-9       # marginal stopping tolerance (l1)
    tol_gap: float = 0.0         # certified relative gap; 0 disables the test
    gap_every: int = 1           # certificate cadence (outer iterations)
    cg_rtol: float = 1e-6        # truncated-CG relative residual
    max_cg: int = 1000           # CG cap (also capped by m + n)
    beta: float = 0.5            # Armijo backtracking factor
    c1: float = 1e-4             # Armijo sufficient-increase constant
    max_backtrack: int = 30
    gamma: float = 1.0           # sparsify budget multiplier (R5)
    sinkhorn_check_every: int = 10


# --------------------------------------------------------------------------- #
# Shifted-cost primal map, Eq. eppa_x with the accumulated potentials (*)
# --------------------------------------------------------------------------- #
def key_matrix(C, F, G, eta, s):
    """eta * log X~ = F_i + G_j - s (C_ij + eta), Eq. eppa_x in form (*)."""
    return (F[:, None] + G[None, :]) - s * (C + eta)


def log_plan(C, F, G, eta, s):
    """log X~^k, Eq. eppa_x in form (*)."""
    return key_matrix(C, F, G, eta, s) / eta


def plan(C, F, G, eta, s):
    """X~^k, Eq. eppa_x in form (*)."""
    return np.exp(log_plan(C, F, G, eta, s))


def logsumexp(Z, axis):
    """Max-shifted log-sum-exp along one axis."""
    mx = np.max(Z, axis=axis, keepdims=True)
    out = mx + np.log(np.sum(np.exp(Z - mx), axis=axis, keepdims=True))
    return np.squeeze(out, axis=axis)


# --------------------------------------------------------------------------- #
# Sinkhorn half-steps, Algorithm 2 warm-up loop (log-domain form of Algorithm 1)
# --------------------------------------------------------------------------- #
def sinkhorn_row_step(C, a, F, G, eta, s):
    """f <- f + eta (log a - log(X~ 1)).  Returns (new F, row residual
    ||X~ 1 - a||_1 measured before the update)."""
    Z = log_plan(C, F, G, eta, s)
    log_r = logsumexp(Z, axis=1)
    res = float(np.sum(np.abs(np.exp(log_r) - a)))
    return F + eta * (np.log(a) - log_r), res


def sinkhorn_col_step(C, b, F, G, eta, s):
    """g <- g + eta (log b - log(X~^T 1)), using the current (new) F."""
    Z = log_plan(C, F, G, eta, s)
    log_c = logsumexp(Z, axis=0)
    return G + eta * (np.log(b) - log_c)


# --------------------------------------------------------------------------- #
# Dual objective, gradient and Hessian of the subproblem, Eqs. eppa-sub-dual,
# eq:eppa-hess and the gradient formulas between them
# --------------------------------------------------------------------------- #
def dual_objective(C, a, b, F, G, eta, s, Phi=None, Psi=None):
    """P^k(f, g) = <a, f> + <b, g> - eta <E, X~^k(f, g)>, with f = F - Phi."""
    f = F if Phi is None else F - Phi
    g = G if Psi is None else G - Psi
    return float(a @ f + b @ g - eta * np.sum(plan(C, F, G, eta, s)))


def marginals(C, F, G, eta, s):
    X = plan(C, F, G, eta, s)
    return X.sum(axis=1), X.sum(axis=0)


def gradient(C, a, b, F, G, eta, s):
    """(grad_f, grad_g) = (a - X~ 1, b - X~^T 1), and the row/column sums."""
    r, c = marginals(C, F, G, eta, s)
    return a - r, b - c, r, c


def dense_hessian(C, F, G, eta, s):
    """Eq. eq:eppa-hess: -(1/eta) [[diag(X~1), X~], [X~^T, diag(X~^T 1)]]."""
    X = plan(C, F, G, eta, s)
    m, n = X.shape
    H = np.zeros((m + n, m + n))
    H[:m, :m] = np.diag(X.sum(axis=1))
    H[m:, m:] = np.diag(X.sum(axis=0))
    H[:m, m:] = X
    H[m:, :m] = X.T
    return -H / eta


def residual_l1(a, b, r, c):
    """R8: ||X~1 - a||_1 + ||X~^T 1 - b||_1."""
    return float(np.sum(np.abs(r - a)) + np.sum(np.abs(c - b)))


# --------------------------------------------------------------------------- #
# Sparsify (Alg. 2; Section 3.2 implementation details; Theorem 2 density)
# --------------------------------------------------------------------------- #
@dataclasses.dataclass
class CSR:
    m: int
    n: int
    indptr: np.ndarray    # int64, m + 1
    indices: np.ndarray   # int64 column of each kept entry
    data: np.ndarray      # float64 value X~_ij

    @property
    def nnz(self):
        return int(self.indices.shape[0])

    def dense(self):
        S = np.zeros((self.m, self.n))
        for i in range(self.m):
            lo, hi = self.indptr[i], self.indptr[i + 1]
            S[i, self.indices[lo:hi]] = self.data[lo:hi]
        return S

    def scipy(self):
        from scipy.sparse import csr_matrix
        return csr_matrix((self.data, self.indices, self.indptr), shape=(self.m, self.n))


def sparsify_budget(m, n, gamma=1.0):
    """R5: number of coupling-block entries kept, K = round(gamma (m + n - 1))."""
    return int(min(m * n, max(1, round(gamma * (m + n - 1)))))


def sparsify(C, F, G, eta, s, K):
    """Keep the K largest X~_ij (ranked by eta log X~ = key, ties -> lower i*n+j),
    returned in CSR row-major order with values X~_ij."""
    m, n = C.shape
    key = key_matrix(C, F, G, eta, s).ravel()
    lin = np.arange(m * n)
    order = np.lexsort((lin, -key))          # key descending, then index ascending
    keep = np.sort(order[:K])
    rows, cols = keep // n, keep % n
    indptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(indptr, rows + 1, 1)
    indptr = np.cumsum(indptr)
    data = np.exp(key[keep] / eta)
    return CSR(m, n, indptr, cols.astype(np.int64), data)


def sparse_matvec(r, c, S, eta, x, y):
    """M (x; y) with M = (1/eta) [[diag r, S], [S^T, diag c]] = -Sparsify(Hessian).
    S may be a CSR (above) or a scipy sparse matrix built from one."""
    Sm = S.scipy() if isinstance(S, CSR) else S
    return (r * x + Sm @ y) / eta, (Sm.T @ x + c * y) / eta


# --------------------------------------------------------------------------- #
# Truncated CG on the sparsified Newton system (Alg. 2; Section 3.2; E.1)
# --------------------------------------------------------------------------- #
def pcg(r, c, S, eta, rhs_f, rhs_g, rtol=1e-6, max_iter=1000):
    """Jacobi-preconditioned CG (Nocedal & Wright, Alg. 5.3) for M d = rhs.
    Returns (d_f, d_g, iterations, final relative residual)."""
    m = r.shape[0]
    rhs = np.concatenate([rhs_f, rhs_g])
    dinv = eta / np.concatenate([r, c])
    Sm = S.scipy()

    def M(v):
        u, w = sparse_matvec(r, c, Sm, eta, v[:m], v[m:])
        return np.concatenate([u, w])

    x = np.zeros_like(rhs)
    res = rhs.copy()
    bnorm = float(np.linalg.norm(rhs))
    if bnorm == 0.0:
        return x[:m], x[m:], 0, 0.0
    z = dinv * res
    p = z.copy()
    rz = float(res @ z)
    it = 0
    rel = 1.0
    while it < max_iter:
        q = M(p)
        alpha = rz / float(p @ q)
        x = x + alpha * p
        res = res - alpha * q
        it += 1
        rel = float(np.linalg.norm(res)) / bnorm
        if rel <= rtol:
            break
        z = dinv * res
        rz_new = float(res @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x[:m], x[m:], it, rel


# --------------------------------------------------------------------------- #
# Armijo backtracking on P^k (Alg. 2; E.1: beta = 0.5, c1 = 1e-4)
# --------------------------------------------------------------------------- #
def objective_increase(C, a, b, F, G, eta, s, df, dg, alpha):
    """P^k(x + alpha d) - P^k(x), evaluated without cancellation (R7)."""
    X = plan(C, F, G, eta, s)
    W = (df[:, None] + dg[None, :]) * (alpha / eta)
    with np.errstate(over="ignore", invalid="ignore"):
        t = np.sum(X * np.expm1(W))
    if not np.isfinite(t):
        return -np.inf
    return float(alpha * (a @ df + b @ dg) - eta * t)


def armijo(C, a, b, F, G, eta, s, df, dg, gtd, beta, c1, max_backtrack):
    """Largest alpha = beta^q, q <= max_backtrack, with sufficient increase.
    Returns (alpha, accepted, trials)."""
    alpha = 1.0
    for q in range(max_backtrack + 1):
        if objective_increase(C, a, b, F, G, eta, s, df, dg, alpha) >= c1 * alpha * gtd:
            return alpha, True, q + 1
        alpha *= beta
    return 0.0, False, max_backtrack + 1


# --------------------------------------------------------------------------- #
# Certified gap (R9): LP weak duality and a feasible rounding
# --------------------------------------------------------------------------- #
def dual_lower_bound(C, a, b, F, eta, s):
    """LP weak duality.  u = F/s - eta; v_j = min_i (C_ij - u_i) (c-transform),
    then u'_i = min_j (C_ij - v_j) >= u_i; <a,u'> + <b,v> <= OPT."""
    u = F / s - eta
    v = np.min(C - u[:, None], axis=0)
    u2 = np.min(C - v[None, :], axis=1)
    return float(a @ u2 + b @ v)


def support_edges(C, F, G, eta, s, count):
    """The `count` largest entries of X~ (key eta log X~ descending, ties -> lower
    linear index i*n+j), as (keys, rows, cols) in that order."""
    m, n = C.shape
    key = key_matrix(C, F, G, eta, s).ravel()
    lin = np.arange(m * n)
    order = np.lexsort((lin, -key))[:count]
    return key[order], order // n, order % n


def support_tree_duals(C, F, G, eta, s, count=None):
    """Support-tree dual (reading R9 (ii)).  Kruskal's maximum-weight spanning
    forest over the `count` (default 2(m + n - 1)) largest plan entries, taken
    in key order; nodes are the rows 0..m-1 and the columns m..m+n-1.  Each tree
    is rooted at its lowest node, which keeps its entropic potential (rows
    u_i = F_i/s - eta, columns v_j = G_j/s); every other node takes the value
    that makes its tree edge tight, u_i + v_j = C_ij.  Returns (u, v, number of
    trees)."""
    m, n = C.shape
    if count is None:
        count = min(m * n, 2 * (m + n - 1))
    _, rows, cols = support_edges(C, F, G, eta, s, count)
    parent = list(range(m + n))

    def find(x):
        while parent[x] != x:
            x = parent[x]
        return x

    adj = [[] for _ in range(m + n)]
    for i, j in zip(rows.tolist(), cols.tolist()):
        ri, rj = find(i), find(m + j)
        if ri != rj:
            parent[max(ri, rj)] = min(ri, rj)
            adj[i].append(m + j)
            adj[m + j].append(i)
    u = np.empty(m)
    v = np.empty(n)
    seen = [False] * (m + n)
    trees = 0
    for root in range(m + n):              # increasing node order: roots are lowest
        if seen[root]:
            continue
        trees += 1
        if root < m:
            u[root] = F[root] / s - eta
        else:
            v[root - m] = G[root - m] / s
        seen[root] = True
        stack = [root]
        while stack:
            x = stack.pop()
            for y in adj[x]:
                if seen[y]:
                    continue
                seen[y] = True
                if x < m:
                    v[y - m] = C[x, y - m] - u[x]
                else:
                    u[y] = C[y, x - m] - v[x - m]
                stack.append(y)
    return u, v, trees


def c_transform_bound(C, a, b, u):
    """LP weak duality for any row potential u: v_j = min_i (C_ij - u_i), then
    u'_i = min_j (C_ij - v_j) >= u_i; (u', v) is dual feasible, so
    <a, u'> + <b, v> <= OPT."""
    v = np.min(C - u[:, None], axis=0)
    u2 = np.min(C - v[None, :], axis=1)
    return float(a @ u2 + b @ v)


def round_to_polytope(X, a, b):
    """Altschuler, Weed & Rigollet (2017), Algorithm 2: scale rows down to a,
    columns down to b, then add err_r err_c^T / ||err_r||_1."""
    x = np.minimum(a / X.sum(axis=1), 1.0)
    X1 = X * x[:, None]
    y = np.minimum(b / X1.sum(axis=0), 1.0)
    X2 = X1 * y[None, :]
    er = a - X2.sum(axis=1)
    ec = b - X2.sum(axis=0)
    l1 = float(np.sum(np.abs(er)))
    if l1 > 0.0:
        X2 = X2 + np.outer(er, ec) / l1
    return X2


def certificate(C, a, b, F, G, eta, s):
    """Returns dict(cost=<C,X~>, lb, ub, rel_gap, lb_entropic, lb_tree)."""
    X = plan(C, F, G, eta, s)
    cost = float(np.sum(C * X))
    ub = float(np.sum(C * round_to_polytope(X, a, b)))
    lb_e = dual_lower_bound(C, a, b, F, eta, s)
    u_t, _, _ = support_tree_duals(C, F, G, eta, s)
    lb_t = c_transform_bound(C, a, b, u_t)
    lb = max(lb_e, lb_t)
    rel = (ub - lb) / lb if lb > 0.0 else (ub - lb) / max(abs(ub), 1e-300)
    return {"cost": cost, "lb": lb, "ub": ub, "rel_gap": float(rel),
            "lb_entropic": lb_e, "lb_tree": lb_t}


# --------------------------------------------------------------------------- #
# Inner solver of subproblem k (Alg. 2 inner loops) and the outer loop
# --------------------------------------------------------------------------- #
def sinkhorn_warmup(C, a, b, F, G, eta, s, cfg: Config):
    """T1 Gauss-Seidel block ascents (R3, R4).  Returns (F, G, iterations)."""
    t = 0
    while t < cfg.T1:
        F, res_row = sinkhorn_row_step(C, a, F, G, eta, s)
        G = sinkhorn_col_step(C, b, F, G, eta, s)
        t += 1
        if t % cfg.sinkhorn_check_every == 0 and res_row <= cfg.tol_marg:
            break
    return F, G, t


def newton_phase(C, a, b, F, G, eta, s, cfg: Config, stats: dict):
    """Up to T2 damped Newton steps on the sparsified Hessian (Alg. 2)."""
    m, n = C.shape
    K = sparsify_budget(m, n, cfg.gamma)
    max_cg = min(cfg.max_cg, m + n)
    res = None
    for _ in range(cfg.T2):
        ga, gb, r, c = gradient(C, a, b, F, G, eta, s)
        res = residual_l1(a, b, r, c)
        if res <= cfg.tol_marg:
            return F, G, res
        S = sparsify(C, F, G, eta, s, K)
        df, dg, it, _ = pcg(r, c, S, eta, ga, gb, cfg.cg_rtol, max_cg)
        stats["cg_iters"] += it
        gtd = float(ga @ df + gb @ dg)
        alpha, ok, trials = armijo(C, a, b, F, G, eta, s, df, dg, gtd,
                                   cfg.beta, cfg.c1, cfg.max_backtrack)
        stats["ls_trials"] += trials
        stats["newton_iters"] += 1
        if ok:
            F = F + alpha * df
            G = G + alpha * dg
        else:
            stats["ls_failures"] += 1
            F, _ = sinkhorn_row_step(C, a, F, G, eta, s)
            G = sinkhorn_col_step(C, b, F, G, eta, s)
    _, _, r, c = gradient(C, a, b, F, G, eta, s)
    return F, G, residual_l1(a, b, r, c)


def pins(C, a, b, cfg: Optional[Config] = None, **overrides):
    """Algorithm 2 with readings R1-R9.  Returns a dict with the final
    potentials (F, G, s: the plan is exp((F_i + G_j - s (C_ij + eta)) / eta)),
    the transport cost <C, X~>, the certificate and a per-outer-iteration trace."""
    cfg = dataclasses.replace(cfg or Config(), **overrides)
    C = np.asarray(C, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m, n = C.shape
    eta = float(cfg.eta)
    Phi, Psi = np.zeros(m), np.zeros(n)           # R1
    F, G = Phi.copy(), Psi.copy()
    stats = {"sinkhorn_iters": 0, "newton_iters": 0, "cg_iters": 0, "ls_trials": 0,
             "ls_failures": 0}
    trace = []
    cert = None
    k = 0
    while k < cfg.K:
        s = float(k + 1)
        F, G, t1 = sinkhorn_warmup(C, a, b, F, G, eta, s, cfg)
        stats["sinkhorn_iters"] += t1
        F, G, res = newton_phase(C, a, b, F, G, eta, s, cfg, stats)
        X = plan(C, F, G, eta, s)                       # X^{k+1}
        rec = {"k": k, "cost": float(np.sum(C * X)), "res": res, "sinkhorn": t1}
        if cfg.tol_gap > 0.0 and ((k + 1) % cfg.gap_every == 0 or k + 1 == cfg.K):
            cert = certificate(C, a, b, F, G, eta, s)
            rec.update(lb=cert["lb"], ub=cert["ub"], rel_gap=cert["rel_gap"])
        trace.append(rec)
        k += 1
        if cert is not None and cert["rel_gap"] <= cfg.tol_gap and "rel_gap" in rec:
            break
        if k < cfg.K:                                   # outer update, R2
            f, g = F - Phi, G - Psi
            Phi, Psi = F, G
            F, G = F + f, G + g
    s = float(k)
    if cert is None or "rel_gap" not in trace[-1]:
        cert = certificate(C, a, b, F, G, eta, s)
    return {"F": F, "G": G, "s": s, "outer_iters": k, "cost": trace[-1]["cost"],
            "res": trace[-1]["res"], "lb": cert["lb"], "ub": cert["ub"],
            "rel_gap": cert["rel_gap"], "trace": trace, **stats}


# --------------------------------------------------------------------------- #
# Plain log-domain Sinkhorn at fixed regularisation (Algorithm 1); the paper's
# "Sinkhorn (no EPPA)" baseline (Section 5.1.1; E.1 cap 50 000, tol 1e-9)
# --------------------------------------------------------------------------- #
def sinkhorn(C, a, b, eps, max_iter=50000, tol=1e-9, f=None, g=None):
    """Algorithm 1 on X(f, g) = exp((f 1^T + 1 g^T - C - eps E)/eps) (Eq. eq:sink_x).
    Returns (f, g, iterations, residual)."""
    m, n = C.shape
    f = np.zeros(m) if f is None else f.copy()
    g = np.zeros(n) if g is None else g.copy()
    res = np.inf
    it = 0
    while it < max_iter:
        Z = (f[:, None] + g[None, :] - C - eps) / eps
        f = f + eps * (np.log(a) - logsumexp(Z, axis=1))
        Z = (f[:, None] + g[None, :] - C - eps) / eps
        g = g + eps * (np.log(b) - logsumexp(Z, axis=0))
        it += 1
        Z = (f[:, None] + g[None, :] - C - eps) / eps
        res = float(np.sum(np.abs(np.exp(logsumexp(Z, axis=1)) - a)))
        if res <= tol:
            break
    return f, g, it, res


def sinkhorn_plan(C, f, g, eps):
    """Eq. eq:sink_x."""
    return np.exp((f[:, None] + g[None, :] - C - eps) / eps)
