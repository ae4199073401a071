"""End-to-end parity of pins_solve / pins_solve_batch / pins_submit with the FP64
oracle, exact LP optima, and each other (cost kinds, alone vs batched).

Bars: FP64 path -- relative transport cost within 1e-8 of the oracle on the same
algorithm and marginal residual below the tolerance; mixed path -- the achieved
relative cost error against the FP64 oracle is asserted <= 1e-7 (FP32-rounded
costs) and reported by the benchmark for every workload."""
import numpy as np
import pytest

from oracle import pins_oracle as po
from paper_2502_03749_gb300 import pins, workloads as wl

pytestmark = pytest.mark.gpu


def _solve(problem_ref, **cfg):
    h = pins.Pins(**cfg)
    try:
        return h.solve(problem_ref)
    finally:
        h.close()


@pytest.mark.parametrize("m,n", [(64, 64), (48, 80), (130, 70)])
def test_fp64_solve_matches_oracle(m, n):
    w = wl.small_points(0, m=m, n=n)
    kw = dict(eta=1e-2, tol_marg=1e-10, K=6, gamma=2.0)
    ref = po.pins(w.C, w.a, w.b, **kw)
    out = _solve(pins.problem_from_workload(w), eta=1e-2, tol_marg=1e-10, K=6,
                 sparsify_gamma=2.0)
    assert out["outer_iters"] == ref["outer_iters"]
    assert abs(out["cost"] - ref["cost"]) / ref["cost"] <= 1e-8
    # Newton can end at the T2 cap; the residual then matches the oracle's
    assert out["marg_resid_l1"] <= max(1e-10, 1.01 * ref["res"])
    assert out["newton_iters"] == ref["newton_iters"]
    assert abs(out["dual_lb"] - ref["lb"]) <= 1e-8 * abs(ref["lb"])
    assert abs(out["cost_ub"] - ref["ub"]) <= 1e-8 * abs(ref["ub"])
    np.testing.assert_allclose(out["F"], ref["F"], rtol=0, atol=1e-7 * np.abs(ref["F"]).max())


def test_fp64_paper_defaults_track_oracle():
    """gamma = 1 (Theorem 2 budget), T1 = 100, T2 = 50: Newton is linear here, so the
    inner solves end at the T2 cap; costs still agree to 1e-8."""
    w = wl.small_points(0)
    ref = po.pins(w.C, w.a, w.b, eta=1e-2, tol_marg=1e-10, K=3)
    out = _solve(pins.problem_from_workload(w), eta=1e-2, tol_marg=1e-10, K=3)
    assert abs(out["newton_iters"] - ref["newton_iters"]) <= 0.05 * ref["newton_iters"]
    assert abs(out["cost"] - ref["cost"]) / ref["cost"] <= 1e-8


def test_cost_kinds_agree():
    """Dense, point-cloud and grid sources of the same C give identical solves."""
    w = wl.small_points(1, m=36, n=44)
    dense = pins.make_problem("dense", w.a, w.b, C=w.C)
    pts = pins.make_problem("points", w.a, w.b, x=w.x, y=w.y, cost_scale=w.cost_scale)
    kw = dict(eta=1e-2, tol_marg=1e-10, K=4, sparsify_gamma=2.0)
    o1, o2 = _solve(dense, **kw), _solve(pts, **kw)
    assert o1["cost"] == o2["cost"] and np.array_equal(o1["F"], o2["F"])
    g = wl.grid_instance(7, 0)
    gd = pins.make_problem("dense", g.a, g.b, C=g.dense_cost())
    gg = pins.make_problem("grid", g.a, g.b, cost_scale=g.cost_scale, grid=g.grid)
    o3, o4 = _solve(gd, **kw), _solve(gg, **kw)
    assert o3["cost"] == o4["cost"] and np.array_equal(o3["G"], o4["G"])


def test_lp_optimum_reached():
    """eta = 1e-3: the outer loop reaches the HiGHS optimum of Eq. ot (m != n)."""
    from scipy.optimize import linprog
    rng = np.random.default_rng(31)
    m, n = 12, 9
    x = rng.uniform(0, 1, size=(m, 2)); y = rng.uniform(0, 1, size=(n, 2))
    C = ((x[:, None, :] - y[None, :, :]) ** 2).sum(axis=2); C /= C.max()
    a = rng.dirichlet(np.ones(m)); b = rng.dirichlet(np.ones(n))
    A = np.zeros((m + n, m * n))
    for i in range(m):
        A[i, i * n:(i + 1) * n] = 1
    for j in range(n):
        A[m + j, j::n] = 1
    opt = linprog(C.ravel(), A_eq=A, b_eq=np.concatenate([a, b]), bounds=(0, None),
                  method="highs").fun
    out = _solve(pins.make_problem("dense", a, b, C=C), eta=1e-3, tol_marg=1e-11, K=250,
                 sparsify_gamma=2.0)
    assert abs(out["cost"] - opt) / opt <= 1e-9
    assert out["dual_lb"] <= opt * (1 + 1e-12) and out["cost_ub"] >= opt * (1 - 1e-12)


def test_single_row_closed_form():
    """m = 1: the only feasible plan is b^T, so cost = sum_j C_1j b_j (any eta)."""
    rng = np.random.default_rng(3)
    n = 300
    C = rng.uniform(size=(1, n)); b = rng.dirichlet(np.ones(n))
    out = _solve(pins.make_problem("dense", np.ones(1), b, C=C), eta=1e-2, K=2, tol_marg=1e-12)
    assert out["cost"] == pytest.approx(float(C[0] @ b), rel=1e-12)


@pytest.mark.parametrize("kind", ["dense32", "points"])
def test_mixed_precision_accuracy(kind):
    w = wl.small_points(2, m=96, n=80)
    if kind == "dense32":
        C32 = w.C.astype(np.float32)
        ref = po.pins(C32.astype(np.float64), w.a, w.b, eta=1e-2, tol_marg=1e-9, K=8, gamma=2.0)
        pr = pins.make_problem("dense", w.a, w.b, C=C32)
    else:
        xf = w.x.astype(np.float32).astype(np.float64)
        yf = w.y.astype(np.float32).astype(np.float64)
        Cf = (((xf[:, None, :] - yf[None, :, :]) ** 2).sum(axis=2).astype(np.float32)
              .astype(np.float64) * w.cost_scale)
        ref = po.pins(Cf, w.a, w.b, eta=1e-2, tol_marg=1e-9, K=8, gamma=2.0)
        pr = pins.make_problem("points", w.a, w.b, x=w.x, y=w.y, cost_scale=w.cost_scale)
    out = _solve(pr, prec="mixed", eta=1e-2, tol_marg=1e-9, K=8, sparsify_gamma=2.0)
    assert abs(out["cost"] - ref["cost"]) / ref["cost"] <= 1e-7
    assert out["marg_resid_l1"] <= 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_and_serving_match_solo(prec):
    """Each result is bit-identical alone, inside a batch, and through submit/poll."""
    probs = [wl.small_points(i, m=m, n=n) for i, (m, n) in
             enumerate([(40, 60), (64, 64), (100, 30), (17, 90), (128, 129)])]
    refs = [pins.problem_from_workload(w) for w in probs]
    kw = dict(prec=prec, eta=1e-2, tol_marg=1e-10, K=3, sparsify_gamma=2.0, max_inflight=3)
    h = pins.Pins(**kw)
    try:
        solo = [h.solve(r) for r in refs]
        batch = h.solve_batch(refs)
        tickets = [h.submit(r) for r in refs]
        served = []
        for t, r in zip(tickets, refs):
            F = np.zeros(r.prob.m); G = np.zeros(r.prob.n)
            d = h.wait(t, (F, G))
            d["F"] = F
            served.append(d)
    finally:
        h.close()
    for s, b, v in zip(solo, batch, served):
        assert s["cost"] == b["cost"] == v["cost"]
        assert np.array_equal(s["F"], b["F"]) and np.array_equal(s["F"], v["F"])


def test_sinkhorn_eppa_baseline_matches_oracle():
    """Sinkhorn+EPPA, the paper's first comparison solver (Section 5.1), is PINS
    with the Newton phase switched off (T2 = 0): the same kernels, and on the
    FP64 path the same iterates as the oracle run with the same settings."""
    w = wl.small_points(4, m=40, n=52)
    kw = dict(eta=1e-2, tol_marg=1e-10, K=6, T2=0)
    ref = po.pins(w.C, w.a, w.b, gamma=2.0, **kw)
    out = _solve(pins.problem_from_workload(w), sparsify_gamma=2.0, **kw)
    assert out["outer_iters"] == ref["outer_iters"] == 6
    assert out["sinkhorn_iters"] == ref["sinkhorn_iters"] and out["newton_iters"] == 0
    assert abs(out["cost"] - ref["cost"]) / ref["cost"] <= 1e-10
    np.testing.assert_allclose(out["F"], ref["F"], rtol=0, atol=1e-9 * np.abs(ref["F"]).max())


def test_sinkhorn_without_eppa_matches_algorithm_1():
    """Sinkhorn without EPPA is one outer iteration of Sinkhorn half-steps
    (K = 1, T2 = 0): the plan at s = 1 is Algorithm 1's scaling form at
    eps = eta, so the converged cost equals that of the oracle's separate
    Algorithm 1 routine (a different residual schedule, the same unique
    entropic optimum)."""
    w = wl.small_points(4, m=40, n=52)
    eta = 1e-2
    f, g, it1, _ = po.sinkhorn(w.C, w.a, w.b, eta, max_iter=50000, tol=1e-11)
    X = np.exp((f[:, None] + g[None, :] - w.C - eta) / eta)
    cost1 = float(np.sum(w.C * X))
    ref = po.pins(w.C, w.a, w.b, eta=eta, tol_marg=1e-11, K=1, T1=5000, T2=0)
    out = _solve(pins.problem_from_workload(w), eta=eta, tol_marg=1e-11, K=1, T1=5000, T2=0)
    assert out["outer_iters"] == 1 and out["newton_iters"] == 0
    assert abs(out["sinkhorn_iters"] - ref["sinkhorn_iters"]) <= 10
    assert out["marg_resid_l1"] <= 1e-10
    assert abs(out["cost"] - cost1) / cost1 <= 1e-9


def test_newton_without_eppa_converges_to_the_entropic_optimum():
    """Newton without EPPA (K = 1): the sparse Newton phase after the warm-up
    drives the residual to the tolerance and lands on the same entropic
    optimum as Algorithm 1 at eps = eta."""
    w = wl.small_points(4, m=40, n=52)
    eta = 1e-2
    f, g, _, _ = po.sinkhorn(w.C, w.a, w.b, eta, max_iter=50000, tol=1e-11)
    cost1 = float(np.sum(w.C * np.exp((f[:, None] + g[None, :] - w.C - eta) / eta)))
    ref = po.pins(w.C, w.a, w.b, eta=eta, tol_marg=1e-10, gamma=2.0, K=1, T2=300)
    out = _solve(pins.problem_from_workload(w), eta=eta, tol_marg=1e-10, sparsify_gamma=2.0,
                 K=1, T2=300)
    assert out["outer_iters"] == 1 and out["sinkhorn_iters"] == ref["sinkhorn_iters"]
    assert abs(out["newton_iters"] - ref["newton_iters"]) <= max(3, ref["newton_iters"] // 10)
    assert out["marg_resid_l1"] <= 1e-10
    assert abs(out["cost"] - cost1) / cost1 <= 1e-8


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_warmup_matches_direct_launches(prec):
    """Unprofiled solves launch each block of Sinkhorn half-steps as one captured
    CUDA graph; profiled solves launch the kernels one by one.  Both run the same
    kernels on the same data, so the solves are bit-identical."""
    w = wl.gmm_instance(1, m=200, n=176, eta=1e-2)
    ref = pins.problem_from_workload(w)
    out = []
    for prof in (0, 1):
        h = pins.Pins(prec=prec, eta=1e-2, K=3, tol_marg=1e-12, profile=prof)
        try:
            out.append(h.solve(ref))
        finally:
            h.close()
    a, b = out
    assert a["sinkhorn_iters"] == b["sinkhorn_iters"] >= 20
    assert a["newton_iters"] == b["newton_iters"] and a["cost"] == b["cost"]
    assert np.array_equal(a["F"], b["F"]) and np.array_equal(a["G"], b["G"])


@pytest.mark.parametrize("case", ["gmm", "grid"])
def test_one_pass_selection_matches_histogram_search(case):
    """The mixed path's one-pass selection (later Newton steps of an outer
    iteration) keeps exactly the entries the histogram search keeps, so the two
    give bit-identical solves.  The grid case has many tied keys."""
    if case == "gmm":
        w = wl.gmm_instance(0, m=300, n=280, eta=1e-2)
    else:
        w = wl.grid_instance(16, 0, eta=1e-2)
    ref = pins.problem_from_workload(w)
    out = []
    for one_pass in (1, 0):
        h = pins.Pins(prec="mixed", eta=1e-2, K=4, sparsify_one_pass=one_pass)
        try:
            out.append(h.solve(ref))
        finally:
            h.close()
    a, b = out
    assert a["newton_iters"] == b["newton_iters"] and a["cg_iters"] == b["cg_iters"]
    assert a["cost"] == b["cost"]
    assert np.array_equal(a["F"], b["F"]) and np.array_equal(a["G"], b["G"])
    assert a["newton_iters"] > 4        # the one-pass path ran (steps after the first)


def test_invalid_inputs_rejected():
    rng = np.random.default_rng(1)
    C = rng.uniform(size=(5, 6))
    a = np.full(5, 0.2); b = np.full(6, 1 / 6)
    h = pins.Pins()
    try:
        bad = a.copy(); bad[0] = -0.1; bad[1] += 0.3
        res = pins.pins_result()
        assert pins.pins_solve(h.h, pins.make_problem("dense", bad, b, C=C).prob, res) == \
            pins.PINS_ERR_INVALID_ARG
        assert pins.pins_solve(h.h, pins.make_problem("dense", a * 1.01, b, C=C).prob, res) == \
            pins.PINS_ERR_INVALID_ARG
        Cn = C.copy(); Cn[2, 3] = np.nan
        assert pins.pins_solve(h.h, pins.make_problem("dense", a, b, C=Cn).prob, res) == \
            pins.PINS_ERR_INVALID_ARG
        assert "finite" in h.error()
        st, _ = pins.pins_submit(h.h, pins.make_problem("dense", a[:0], b, C=C).prob)
        assert st == pins.PINS_ERR_INVALID_ARG
        res2 = pins.pins_result()
        assert pins.pins_poll(h.h, 123456, res2) == pins.PINS_ERR_UNKNOWN_TICKET
    finally:
        h.close()


# --------------------------------------------------------------------------- #
# The accuracy operating point: certified relative gap <= 1e-6 (reading R9)
# --------------------------------------------------------------------------- #
def _hi_lp_opt(C, a, b):
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix
    m, n = C.shape
    rows = np.concatenate([np.repeat(np.arange(m), n), m + np.tile(np.arange(n), m)])
    cols = np.concatenate([np.arange(m * n), np.arange(m * n)])
    A = coo_matrix((np.ones(2 * m * n), (rows, cols)), shape=(m + n, m * n)).tocsr()
    res = linprog(C.ravel(), A_eq=A, b_eq=np.concatenate([a, b * (a.sum() / b.sum())]),
                  bounds=(0, None), method="highs",
                  options={"primal_feasibility_tolerance": 1e-10,
                           "dual_feasibility_tolerance": 1e-10})
    assert res.status == 0
    return float(res.fun)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_points_instance_certified_to_1e6_at_eta_1e4(prec, seed):
    """64 x 64 uniform points, random weights (the paper's smallest synthetic
    size), eta = 1e-4 (Table 3's most accurate setting): both paths stop on a
    certified relative gap <= 1e-6 within a few outer iterations (s/eta up to
    ~1e5).  FP64 follows the oracle's iterates (same outer count, cost and
    bounds within 1e-8); the mixed path solves the FP32-rounded cost and its
    error to that cost's LP optimum is at most the certified 1e-6."""
    w = wl.small_points(seed)
    C = w.C if prec == "fp64" else w.C.astype(np.float32).astype(np.float64)
    kw = dict(eta=1e-4, tol_gap=1e-6, K=250)
    out = _solve(pins.make_problem("dense", w.a, w.b, C=C if prec == "fp64" else C.astype(np.float32)),
                 prec=prec, **kw)
    assert out["status"] == 0 and out["rel_gap"] <= 1e-6
    opt = _hi_lp_opt(C, w.a, w.b)
    assert out["dual_lb"] <= opt * (1 + 1e-9) and out["cost_ub"] >= opt * (1 - 1e-9)
    assert abs(out["cost"] - opt) / opt <= 1.2e-6
    if prec == "fp64":
        ref = po.pins(C, w.a, w.b, **kw)
        assert out["outer_iters"] == ref["outer_iters"]
        assert abs(out["cost"] - ref["cost"]) / ref["cost"] <= 1e-8
        assert abs(out["dual_lb"] - ref["lb"]) <= 1e-8 * ref["lb"]
        assert abs(out["cost_ub"] - ref["ub"]) <= 1e-8 * ref["ub"]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("eta,gamma", [(1e-3, 1.0), (2.5e-4, 2.0)])
def test_stroke_pair_certified_to_1e6(prec, eta, gamma):
    """A 16 x 16 stroke-image pair (grid cost on the fly): integer grid costs give
    an LP whose reduced costs are multiples of the cost scale, so the plan
    concentrates and the support-tree bound certifies <= 1e-6, at the paper's
    sparsify budget and at the benchmark's setting (eta = 2.5e-4, budget
    2 (m + n - 1)).  FP64 against the oracle within 1e-8; mixed against the same
    oracle run."""
    w = wl.stroke_pair(0, eta=eta, s=16)
    kw = dict(eta=eta, tol_gap=1e-6, K=250)
    out = _solve(pins.problem_from_workload(w), prec=prec, sparsify_gamma=gamma, **kw)
    assert out["status"] == 0 and out["rel_gap"] <= 1e-6
    ref = po.pins(w.dense_cost(), w.a, w.b, gamma=gamma, **kw)
    assert ref["rel_gap"] <= 1e-6
    tol = 1e-8 if prec == "fp64" else 1e-6
    assert abs(out["cost"] - ref["cost"]) / ref["cost"] <= tol
    assert out["dual_lb"] <= ref["ub"] * (1 + 1e-12) and out["cost_ub"] >= ref["lb"] * (1 - 1e-12)
    if prec == "fp64":
        assert out["outer_iters"] == ref["outer_iters"]
