"""Parity of each hot-path step (through the C ABI step entry points) with the
FP64 oracle on identical inputs.  Sizes span several 64 x 128 tiles, a ragged
tail, and the degenerate 1 x n / m x 1 shapes.

Tolerances: FP64 path -- rounding of FP64 sums and exp (1e-12 relative on sums);
mixed path -- the double-float exp/exponent (~1e-13 relative per entry, 1e-10 on
sums), and FP32 exp in the Sinkhorn warm-up (1e-6 relative per term)."""
import numpy as np
import pytest

from oracle import pins_oracle as po
from paper_2502_03749_gb300 import pins

from gpu_util import dense_device_problem, dev, random_state

pytestmark = pytest.mark.gpu

SHAPES = [(70, 150), (200, 333), (1, 37), (129, 1), (64, 64)]
PRECS = ["fp64", "mixed"]


@pytest.fixture(scope="module")
def handles():
    hs = {p: pins.Pins(prec=p, eta=0.05) for p in PRECS}
    yield hs
    for h in hs.values():
        h.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("m,n", SHAPES)
def test_marginals(handles, prec, m, n):
    import torch
    C, a, b, F, G, eta, s = random_state(m, n, m * 7 + n)
    h = handles[prec]
    prob = dense_device_problem(C.astype(np.float32) if prec == "mixed" else C, a, b)
    r = torch.zeros(m, dtype=torch.float64, device="cuda")
    c = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    st = pins.pins_step_marginals(h.h, prob.prob, s, dev(F), dev(G), r, c, out)
    assert st == 0, h.error()
    _, _, r0, c0 = po.gradient(C, a, b, F, G, eta, s)
    tol = 1e-12 if prec == "fp64" else 1e-10
    np.testing.assert_allclose(r.cpu().numpy(), r0, rtol=tol)
    np.testing.assert_allclose(c.cpu().numpy(), c0, rtol=tol)
    o = out.cpu().numpy()
    assert o[0] == pytest.approx(po.residual_l1(a, b, r0, c0), rel=1e-8, abs=1e-15)
    assert o[1] == pytest.approx(r0.sum(), rel=tol)
    assert o[2] == pytest.approx(po.key_matrix(C, F, G, eta, s).max(), rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("prec", PRECS)
def test_marginals_at_the_benchmark_size(prec):
    """The benchmark's instance (4096 x 4096 GMM, eta = 1e-2) in the launch
    configuration the solver uses at that size: every row and column sum of
    the plan against the oracle on the same cost (FP32-rounded for the mixed
    path), at potentials two Sinkhorn iterations into outer iteration 3."""
    import torch
    from paper_2502_03749_gb300 import workloads as wl
    n = 4096
    w = wl.gmm_instance(0, m=n, n=n, eta=1e-2)
    C = w.C if prec == "fp64" else w.C.astype(np.float32).astype(np.float64)
    eta, s = 1e-2, 3.0
    F, G = np.zeros(n), np.zeros(n)
    for _ in range(2):
        F, _ = po.sinkhorn_row_step(C, w.a, F, G, eta, s)
        G = po.sinkhorn_col_step(C, w.b, F, G, eta, s)
    r = torch.zeros(n, dtype=torch.float64, device="cuda")
    c = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    h = pins.Pins(prec=prec, eta=eta)
    try:
        prob = dense_device_problem(C.astype(np.float32) if prec == "mixed" else C, w.a, w.b)
        st = pins.pins_step_marginals(h.h, prob.prob, s, dev(F), dev(G), r, c, out)
        assert st == 0, h.error()
        torch.cuda.synchronize()
    finally:
        h.close()
    _, _, r0, c0 = po.gradient(C, w.a, w.b, F, G, eta, s)
    tol = 1e-12 if prec == "fp64" else 1e-10
    np.testing.assert_allclose(r.cpu().numpy(), r0, rtol=tol)
    np.testing.assert_allclose(c.cpu().numpy(), c0, rtol=tol)
    assert out.cpu().numpy()[1] == pytest.approx(r0.sum(), rel=tol)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("m,n", SHAPES)
def test_sinkhorn_half_steps(handles, prec, m, n):
    import torch
    C, a, b, F, G, eta, s = random_state(m, n, m * 11 + n)
    F = F * 0.0; G = G * 0.0
    h = handles[prec]
    prob = dense_device_problem(C.astype(np.float32) if prec == "mixed" else C, a, b)
    Fd, Gd = dev(F), dev(G)
    rr = torch.zeros(3, dtype=torch.float64, device="cuda")
    st = pins.pins_step_sinkhorn(h.h, prob.prob, s, 3, Fd, Gd, rr)
    assert st == 0, h.error()
    Fo, Go, res = F.copy(), G.copy(), []
    for _ in range(3):
        Fo, rres = po.sinkhorn_row_step(C, a, Fo, Go, eta, s)
        Go = po.sinkhorn_col_step(C, b, Fo, Go, eta, s)
        res.append(rres)
    atol = 1e-11 if prec == "fp64" else 2e-6 * eta
    np.testing.assert_allclose(Fd.cpu().numpy(), Fo, atol=atol, rtol=0)
    np.testing.assert_allclose(Gd.cpu().numpy(), Go, atol=atol, rtol=0)
    # the mixed warm-up sums FP32 exponentials: its residual floor is ~1e-7
    np.testing.assert_allclose(rr.cpu().numpy(), res, rtol=1e-9 if prec == "fp64" else 1e-4,
                               atol=1e-14 if prec == "fp64" else 2e-7)


GRIDS = [(7, 9), (16, 16), (1, 40), (33, 1), (48, 20), (64, 64)]


def _grid_state(s1, s2, seed, eta):
    """Dirichlet marginals on an s1 x s2 grid, squared grid distance / max, and
    potentials a few eta away from zero."""
    from paper_2502_03749_gb300 import workloads as wl
    rng = np.random.default_rng(seed)
    m = s1 * s2
    a, b = rng.dirichlet(np.ones(m)), rng.dirichlet(np.ones(m))
    scale = 1.0 / max(1, (s1 - 1) ** 2 + (s2 - 1) ** 2)
    w = wl.Problem("grid", a, b, eta, cost_scale=scale, grid=(s1, s2))
    F, G = rng.normal(size=m) * 2 * eta, rng.normal(size=m) * 2 * eta
    return w, F, G


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("s1,s2", GRIDS)
def test_sinkhorn_half_steps_grid(handles, prec, s1, s2):
    """Grid costs generated on the fly.  The mixed path forms each half-step's
    log-sum-exp in two separable stages (over the grid's rows, then its
    columns); both paths against the oracle on the dense cost."""
    import torch
    eta, s = 0.05, 3.0
    w, F, G = _grid_state(s1, s2, s1 * 101 + s2, eta)
    C = w.dense_cost()
    h = handles[prec]
    ad, bd = dev(w.a), dev(w.b)
    prob = pins.make_problem("grid", ad, bd, cost_scale=w.cost_scale, grid=w.grid, on_device=True)
    Fd, Gd = dev(F), dev(G)
    rr = torch.zeros(3, dtype=torch.float64, device="cuda")
    st = pins.pins_step_sinkhorn(h.h, prob.prob, s, 3, Fd, Gd, rr)
    assert st == 0, h.error()
    Fo, Go, res = F.copy(), G.copy(), []
    for _ in range(3):
        Fo, rres = po.sinkhorn_row_step(C, w.a, Fo, Go, eta, s)
        Go = po.sinkhorn_col_step(C, w.b, Fo, Go, eta, s)
        res.append(rres)
    atol = 1e-11 if prec == "fp64" else 2e-6 * eta
    np.testing.assert_allclose(Fd.cpu().numpy(), Fo, atol=atol, rtol=0)
    np.testing.assert_allclose(Gd.cpu().numpy(), Go, atol=atol, rtol=0)
    np.testing.assert_allclose(rr.cpu().numpy(), res, rtol=1e-9 if prec == "fp64" else 1e-4,
                               atol=1e-14 if prec == "fp64" else 2e-7)


def test_sinkhorn_grid_at_the_benchmark_scale():
    """64 x 64 grid at the benchmark's eta = 2.5e-4 and s = 20 (s / eta = 8e4):
    most terms of a row underflow, the kept ones span the full FP32 range of
    2^(w - M).  One mixed iteration against the oracle."""
    import torch
    eta, s = 2.5e-4, 20.0
    w, F, G = _grid_state(64, 64, 77, eta)
    C = w.dense_cost()
    h = pins.Pins(prec="mixed", eta=eta)
    try:
        ad, bd = dev(w.a), dev(w.b)
        prob = pins.make_problem("grid", ad, bd, cost_scale=w.cost_scale, grid=w.grid,
                                 on_device=True)
        Fd, Gd = dev(F), dev(G)
        rr = torch.zeros(1, dtype=torch.float64, device="cuda")
        st = pins.pins_step_sinkhorn(h.h, prob.prob, s, 1, Fd, Gd, rr)
        assert st == 0, h.error()
        Fg, Gg, rg = Fd.cpu().numpy(), Gd.cpu().numpy(), rr.cpu().numpy()
    finally:
        h.close()
    Fo, rres = po.sinkhorn_row_step(C, w.a, F, G, eta, s)
    Go = po.sinkhorn_col_step(C, w.b, Fo, G, eta, s)
    np.testing.assert_allclose(Fg, Fo, atol=2e-6 * eta, rtol=0)
    np.testing.assert_allclose(Gg, Go, atol=2e-6 * eta, rtol=0)
    assert rg[0] == pytest.approx(rres, rel=1e-4, abs=2e-7)


@pytest.mark.parametrize("m,n", [(300, 2048), (1030, 4096)])
def test_sinkhorn_bulk_copy_segments(handles, m, n):
    """Dense FP32 costs whose width is a multiple of 1024 take the row pass that
    streams each row segment through shared memory with bulk async copies."""
    C, a, b, F, G, eta, s = random_state(m, n, m + 3 * n)
    F = F * 0.0; G = G * 0.0
    h = handles["mixed"]
    prob = dense_device_problem(C.astype(np.float32), a, b)
    Fd, Gd = dev(F), dev(G)
    rr = torch_zeros(3)
    st = pins.pins_step_sinkhorn(h.h, prob.prob, s, 3, Fd, Gd, rr)
    assert st == 0, h.error()
    Fo, Go = F.copy(), G.copy()
    for _ in range(3):
        Fo, _ = po.sinkhorn_row_step(C, a, Fo, Go, eta, s)
        Go = po.sinkhorn_col_step(C, b, Fo, Go, eta, s)
    np.testing.assert_allclose(Fd.cpu().numpy(), Fo, atol=2e-6 * eta, rtol=0)
    np.testing.assert_allclose(Gd.cpu().numpy(), Go, atol=2e-6 * eta, rtol=0)


def torch_zeros(k):
    import torch
    return torch.zeros(k, dtype=torch.float64, device="cuda")


def _tie_state(m, n, seed):
    rng = np.random.default_rng(seed)
    C = rng.integers(0, 3, size=(m, n)).astype(np.float64) / 4.0
    F = rng.integers(0, 2, size=m).astype(np.float64) * 0.25
    G = rng.integers(0, 2, size=n).astype(np.float64) * 0.25
    a = np.full(m, 1.0 / m); b = np.full(n, 1.0 / n)
    return C, a, b, F, G, 0.1, 2.0


@pytest.mark.parametrize("case", ["random", "ties"])
@pytest.mark.parametrize("m,n", [(70, 150), (200, 333), (1, 37), (129, 1)])
def test_sparsify_pattern_is_exact_fp64(handles, case, m, n):
    import torch
    if case == "random":
        C, a, b, F, G, eta, s = random_state(m, n, m + 3 * n)
    else:
        C, a, b, F, G, eta, s = _tie_state(m, n, m + 5 * n)
    keep = min(m * n, m + n - 1)
    h = pins.Pins(prec="fp64", eta=eta)
    try:
        prob = dense_device_problem(C, a, b)
        indptr = torch.zeros(m + 1, dtype=torch.int32, device="cuda")
        indices = torch.zeros(keep, dtype=torch.int32, device="cuda")
        data = torch.zeros(keep, dtype=torch.float64, device="cuda")
        st = pins.pins_step_sparsify(h.h, prob.prob, s, dev(F), dev(G), keep, indptr, indices, data)
        assert st == 0, h.error()
    finally:
        h.close()
    S = po.sparsify(C, F, G, eta, s, keep)
    assert np.array_equal(indptr.cpu().numpy(), S.indptr)
    assert np.array_equal(indices.cpu().numpy(), S.indices)
    np.testing.assert_allclose(data.cpu().numpy(), S.data, rtol=1e-14)


@pytest.mark.parametrize("m,n", [(70, 150), (200, 333)])
def test_sparsify_pattern_valid_mixed(handles, m, n):
    """Mixed path ranks by the FP32 value of log X~: the kept set must be a top-K set
    up to that rounding (every kept entry >= every dropped entry within 1e-5)."""
    import torch
    C, a, b, F, G, eta, s = random_state(m, n, 17 * m + n)
    keep = m + n - 1
    prob = dense_device_problem(C.astype(np.float32), a, b)
    indptr = torch.zeros(m + 1, dtype=torch.int32, device="cuda")
    indices = torch.zeros(keep, dtype=torch.int32, device="cuda")
    data = torch.zeros(keep, dtype=torch.float64, device="cuda")
    st = pins.pins_step_sparsify(handles["mixed"].h, prob.prob, s, dev(F), dev(G), keep,
                                 indptr, indices, data)
    assert st == 0, handles["mixed"].error()
    ip, ix = indptr.cpu().numpy(), indices.cpu().numpy()
    assert ip[-1] == keep
    mask = np.zeros((m, n), dtype=bool)
    for i in range(m):
        cols = ix[ip[i]:ip[i + 1]]
        assert np.all(np.diff(cols) > 0)
        mask[i, cols] = True
    Z = po.log_plan(C, F, G, eta, s)
    assert Z[mask].min() >= Z[~mask].max() - 1e-5
    np.testing.assert_allclose(np.sort(data.cpu().numpy()), np.sort(np.exp(Z[mask])), rtol=1e-5)


@pytest.mark.parametrize("m,n", [(70, 150), (40, 40), (1, 9)])
def test_cg_matches_dense_solve(handles, m, n):
    import torch
    C, a, b, F, G, eta, s = random_state(m, n, 5 * m + n)
    ga, gb, r, c = po.gradient(C, a, b, F, G, eta, s)
    S = po.sparsify(C, F, G, eta, s, min(m * n, m + n - 1))
    Sd = S.dense()
    M = np.block([[np.diag(r), Sd], [Sd.T, np.diag(c)]]) / eta
    rhs = np.concatenate([ga, gb])
    # with every entry kept (m = 1 here) M is singular along the gauge direction
    # (e, -e); solutions then differ along it, so compare M d with rhs
    singular = S.nnz == m * n
    d = torch.zeros(m + n, dtype=torch.float64, device="cuda")
    info = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = pins.pins_step_cg(handles["fp64"].h, m, n, eta, dev(r), dev(c),
                           dev(S.indptr.astype(np.int32)), dev(S.indices.astype(np.int32)),
                           dev(S.data), S.nnz, dev(rhs), d, 1e-12, 5000, info)
    assert st == 0, handles["fp64"].error()
    it, rel = info.cpu().numpy()
    assert rel <= 1e-12
    dd_ = d.cpu().numpy()
    assert np.linalg.norm(M @ dd_ - rhs) <= 1e-10 * np.linalg.norm(rhs)
    if not singular:
        want = np.linalg.solve(M, rhs)
        np.testing.assert_allclose(dd_, want, rtol=1e-7, atol=1e-9 * np.abs(want).max())
    dfo, dgo, ito, _ = po.pcg(r, c, S, eta, ga, gb, rtol=1e-12, max_iter=5000)
    assert abs(int(it) - ito) <= max(2, ito // 10)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("alpha", [1.0, 0.25])
def test_objective_increase(handles, prec, alpha):
    m, n = 70, 150
    C, a, b, F, G, eta, s = random_state(m, n, 99)
    rng = np.random.default_rng(5)
    df, dg = rng.normal(size=m) * 1e-3 * eta, rng.normal(size=n) * 1e-3 * eta
    prob = dense_device_problem(C.astype(np.float32) if prec == "mixed" else C, a, b)
    import torch
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = pins.pins_step_objective_increase(handles[prec].h, prob.prob, s, dev(F), dev(G),
                                           dev(df), dev(dg), alpha, out)
    assert st == 0, handles[prec].error()
    want = po.objective_increase(C, a, b, F, G, eta, s, df, dg, alpha)
    scale = alpha * (np.abs(a @ df) + np.abs(b @ dg))
    if prec == "fp64":
        assert abs(out.item() - want) <= 1e-12 * scale + 1e-18
    else:
        # the mixed pass sums the nonnegative terms X~ (expm1(t) - t) in FP32
        # (relative error well below 1e-5); the linear part is FP64
        X = po.plan(C, F, G, eta, s)
        W = (df[:, None] + dg[None, :]) * (alpha / eta)
        R = float(np.sum(X * (np.expm1(W) - W)))
        assert abs(out.item() - want) <= 1e-10 * scale + 1e-5 * eta * R + 1e-18


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("m,n", [(70, 150), (129, 1), (64, 64)])
def test_certificate(handles, prec, m, n):
    import torch
    C, a, b, F, G, eta, s = random_state(m, n, 3 * m + 2 * n)
    prob = dense_device_problem(C.astype(np.float32) if prec == "mixed" else C, a, b)
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    st = pins.pins_step_certificate(handles[prec].h, prob.prob, s, dev(F), dev(G), out)
    assert st == 0, handles[prec].error()
    Cx = C.astype(np.float32).astype(np.float64) if prec == "mixed" else C
    cert = po.certificate(Cx, a, b, F, G, eta, s)
    o = out.cpu().numpy()
    tol = 1e-11 if prec == "fp64" else 1e-9
    assert o[0] == pytest.approx(cert["cost"], rel=tol)
    assert o[1] == pytest.approx(cert["ub"], rel=tol)
    assert o[4] == pytest.approx(cert["lb_entropic"], rel=tol, abs=1e-13)
    assert o[2] == max(o[4], o[5])
    if prec == "fp64":
        # same keys, so the same support, forest and potentials as the oracle
        assert o[5] == pytest.approx(cert["lb_tree"], rel=tol, abs=1e-13)
        assert o[2] == pytest.approx(cert["lb"], rel=tol, abs=1e-13)
    else:
        # the support is selected by FP32 keys: still a valid bound, and close
        assert o[5] <= _lp_opt(Cx, a, b) * (1 + 1e-12) + 1e-15
        assert o[5] == pytest.approx(cert["lb_tree"], rel=1e-6, abs=1e-12)


def _lp_opt(C, a, b):
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix
    m, n = C.shape
    rows = np.concatenate([np.repeat(np.arange(m), n), m + np.tile(np.arange(n), m)])
    cols = np.concatenate([np.arange(m * n), np.arange(m * n)])
    A = coo_matrix((np.ones(2 * m * n), (rows, cols)), shape=(m + n, m * n)).tocsr()
    res = linprog(C.ravel(), A_eq=A, b_eq=np.concatenate([a, b * (a.sum() / b.sum())]),
                  bounds=(0, None), method="highs")
    assert res.status == 0
    return float(res.fun)


def _nw_corner_1d(m, n, seed):
    rng = np.random.default_rng(seed)
    x = np.sort(rng.uniform(0, 1, size=m))
    y = np.sort(rng.uniform(0, 1, size=n))
    a = rng.uniform(0.5, 1.5, size=m); a /= a.sum()
    b = rng.uniform(0.5, 1.5, size=n); b /= b.sum()
    C = (x[:, None] - y[None, :]) ** 2
    C = (C / C.max()).astype(np.float32).astype(np.float64)
    i = j = 0
    ra, rb = a.copy(), b.copy()
    opt = 0.0
    while i < m and j < n:
        t = min(ra[i], rb[j])
        opt += t * C[i, j]
        ra[i] -= t; rb[j] -= t
        if ra[i] <= rb[j]:
            i += 1
        else:
            j += 1
    return C, a, b, opt


@pytest.mark.parametrize("prec", PRECS)
def test_certificate_tree_bound_reaches_the_optimum(handles, prec):
    """On a concentrated plan of a non-degenerate instance (1-D, random weights;
    optimum by the north-west corner rule) the support-tree bound equals OPT to
    rounding on both paths, far above the entropic-dual bound."""
    import torch
    C, a, b, opt = _nw_corner_1d(20, 27, 7)
    eta = 1e-3
    res = po.pins(C, a, b, eta=eta, tol_marg=1e-12, K=8)
    F, G, s = res["F"], res["G"], res["s"]
    prob = dense_device_problem(C.astype(np.float32) if prec == "mixed" else C, a, b)
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    st = pins.pins_step_certificate(handles[prec].h, prob.prob, s, dev(F), dev(G), out)
    assert st == 0, handles[prec].error()
    o = out.cpu().numpy()
    assert abs(o[5] - opt) <= 1e-12 * opt
    assert o[2] == o[5]
    assert opt - o[4] > 1e-6 * opt
    assert o[1] >= opt * (1 - 1e-12)


def test_step_rejects_host_pointers(handles):
    rng = np.random.default_rng(0)
    C = rng.uniform(size=(4, 5)); a = np.full(4, 0.25); b = np.full(5, 0.2)
    pr = pins.make_problem("dense", a, b, C=C)
    import torch
    F = torch.zeros(4, dtype=torch.float64, device="cuda")
    G = torch.zeros(5, dtype=torch.float64, device="cuda")
    assert pins.pins_step_sinkhorn(handles["fp64"].h, pr.prob, 1.0, 1, F, G, None) == \
        pins.PINS_ERR_INVALID_ARG


@pytest.mark.parametrize("m,n,rtol", [(70, 150, 1e-10), (40, 40, 1e-10), (1, 9, 1e-10),
                                      (256, 256, 1e-9), (200, 313, 1e-9), (430, 590, 1e-9),
                                      (700, 1500, 1e-6), (1234, 777, 1e-9)])
def test_cg_double_float_matches_dense_solve(handles, m, n, rtol):
    """The mixed handle runs the CG in double-float arithmetic with FP32 inner
    products: M d must still reproduce rhs to the requested relative residual,
    and the iteration count stays close to the FP64 oracle's.  The sizes cover
    every cluster size: one CTA (up to 512 unknowns, 512 included), 4 CTAs (513
    and 1020 unknowns), 8 (2011) and 16 (2200)."""
    import torch
    C, a, b, F, G, eta, s = random_state(m, n, 7 * m + n)
    ga, gb, r, c = po.gradient(C, a, b, F, G, eta, s)
    S = po.sparsify(C, F, G, eta, s, min(m * n, m + n - 1))
    rhs = np.concatenate([ga, gb])
    d = torch.zeros(m + n, dtype=torch.float64, device="cuda")
    info = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = pins.pins_step_cg(handles["mixed"].h, m, n, eta, dev(r), dev(c),
                           dev(S.indptr.astype(np.int32)), dev(S.indices.astype(np.int32)),
                           dev(S.data), S.nnz, dev(rhs), d, rtol, 5000, info)
    assert st == 0, handles["mixed"].error()
    it, rel = info.cpu().numpy()
    assert rel <= rtol * 1.0001
    dd_ = d.cpu().numpy()
    Sd = S.dense()
    M = np.block([[np.diag(r), Sd], [Sd.T, np.diag(c)]]) / eta
    true_rel = np.linalg.norm(M @ dd_ - rhs) / np.linalg.norm(rhs)
    assert true_rel <= 2.0 * rtol + 1e-12
    if S.nnz < m * n and m + n <= 1500:
        want = np.linalg.solve(M, rhs)
        err = np.linalg.norm(dd_ - want) / np.linalg.norm(want)
        assert err <= max(1e-6, 1e4 * rtol)
    dfo, dgo, ito, _ = po.pcg(r, c, S, eta, ga, gb, rtol=rtol, max_iter=5000)
    assert abs(int(it) - ito) <= max(3, ito // 5)


def test_cg_double_float_is_deterministic(handles):
    import torch
    m, n = 300, 500
    C, a, b, F, G, eta, s = random_state(m, n, 11)
    ga, gb, r, c = po.gradient(C, a, b, F, G, eta, s)
    S = po.sparsify(C, F, G, eta, s, m + n - 1)
    rhs = np.concatenate([ga, gb])
    outs = []
    for _ in range(3):
        d = torch.zeros(m + n, dtype=torch.float64, device="cuda")
        info = torch.zeros(2, dtype=torch.float64, device="cuda")
        st = pins.pins_step_cg(handles["mixed"].h, m, n, eta, dev(r), dev(c),
                               dev(S.indptr.astype(np.int32)), dev(S.indices.astype(np.int32)),
                               dev(S.data), S.nnz, dev(rhs), d, 1e-8, 5000, info)
        assert st == 0
        outs.append(d.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
