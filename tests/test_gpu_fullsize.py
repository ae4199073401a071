"""Parity at the sizes and scales the solves and the benchmark actually reach.

* Mixed-path steps against the oracle at s/eta = 2.5e4 and 2.5e5 (the exponent is
  then formed from terms of size ~s/eta; double-float keeps ~2^-46 of it).
* The double-float CG on systems of 8192 unknowns (16 CTAs x 512), with the
  Theorem 2 budget and twice it, and with so many entries that they live in
  global memory instead of shared memory; the cooperative FP64 CG that systems
  above ~51 000 unknowns fall back to.
* FP64 sparsify against the oracle at 4096 x 4096, and on tied grid keys where
  the threshold bin has to be refined (exact ties resolved by index) or cannot
  be (the documented error).
* The one-pass selection's failure path, forced from the host: the redone
  steps give the same solve bit for bit.
"""
import numpy as np
import pytest

from oracle import pins_oracle as po
from paper_2502_03749_gb300 import pins, workloads as wl

from gpu_util import dense_device_problem, dev, random_state

pytestmark = pytest.mark.gpu


def _zeros(k, dtype=None):
    import torch
    return torch.zeros(k, dtype=dtype or torch.float64, device="cuda")


# --------------------------------------------------------------------------- #
# mixed steps at large s / eta
# --------------------------------------------------------------------------- #
SCALES = [(1e-3, 25.0), (1e-4, 25.0)]     # s / eta = 2.5e4, 2.5e5


@pytest.mark.parametrize("eta,s", SCALES)
def test_mixed_steps_at_large_scale(eta, s):
    """Marginals, Sinkhorn half-steps, objective increase and certificate of the
    mixed path against the oracle on the FP32-rounded cost.  The double-float
    exponent carries an absolute error of about 2^-46 s/eta, so the sums are
    compared at max(1e-10, 4e-14 s/eta) relative."""
    import torch
    m, n = 200, 333
    C, a, b, F, G, eta, s = random_state(m, n, 4242, eta=eta, s=s)
    h = pins.Pins(prec="mixed", eta=eta)
    try:
        prob = dense_device_problem(C.astype(np.float32), a, b)
        tol = max(1e-10, 4e-14 * s / eta)
        # marginals
        r, c, out = _zeros(m), _zeros(n), _zeros(3)
        assert pins.pins_step_marginals(h.h, prob.prob, s, dev(F), dev(G), r, c, out) == 0, h.error()
        _, _, r0, c0 = po.gradient(C, a, b, F, G, eta, s)
        np.testing.assert_allclose(r.cpu().numpy(), r0, rtol=tol)
        np.testing.assert_allclose(c.cpu().numpy(), c0, rtol=tol)
        # Sinkhorn half-steps (FP32 exponentials after the double-float exponent)
        Fd, Gd = dev(F), dev(G)
        assert pins.pins_step_sinkhorn(h.h, prob.prob, s, 2, Fd, Gd, None) == 0, h.error()
        Fo, Go = F.copy(), G.copy()
        for _ in range(2):
            Fo, _ = po.sinkhorn_row_step(C, a, Fo, Go, eta, s)
            Go = po.sinkhorn_col_step(C, b, Fo, Go, eta, s)
        np.testing.assert_allclose(Fd.cpu().numpy(), Fo, atol=2e-6 * eta, rtol=0)
        np.testing.assert_allclose(Gd.cpu().numpy(), Go, atol=2e-6 * eta, rtol=0)
        # objective increase of a small step
        rng = np.random.default_rng(7)
        df, dg = rng.normal(size=m) * 1e-3 * eta, rng.normal(size=n) * 1e-3 * eta
        o1 = _zeros(1)
        assert pins.pins_step_objective_increase(h.h, prob.prob, s, dev(F), dev(G), dev(df),
                                                 dev(dg), 1.0, o1) == 0, h.error()
        want = po.objective_increase(C, a, b, F, G, eta, s, df, dg, 1.0)
        X = po.plan(C, F, G, eta, s)
        W = (df[:, None] + dg[None, :]) / eta
        R = float(np.sum(X * (np.expm1(W) - W)))
        scale = np.abs(a @ df) + np.abs(b @ dg)
        assert abs(o1.item() - want) <= tol * scale + 1e-5 * eta * R + 1e-18
        # certificate
        o6 = _zeros(6)
        assert pins.pins_step_certificate(h.h, prob.prob, s, dev(F), dev(G), o6) == 0, h.error()
        cert = po.certificate(C, a, b, F, G, eta, s)
        o = o6.cpu().numpy()
        assert o[0] == pytest.approx(cert["cost"], rel=10 * tol)
        assert o[1] == pytest.approx(cert["ub"], rel=10 * tol)
        assert o[4] == pytest.approx(cert["lb_entropic"], rel=1e-9, abs=1e-13)
    finally:
        h.close()


@pytest.mark.parametrize("eta,s", SCALES)
def test_mixed_sparsify_valid_at_large_scale(eta, s):
    """The mixed path ranks by the FP32 value of log X~, whose rounding grows
    with s/eta: the kept set is a top-K set up to 2^-22 |log X~|."""
    import torch
    m, n = 200, 333
    C, a, b, F, G, eta, s = random_state(m, n, 4343, eta=eta, s=s)
    keep = m + n - 1
    h = pins.Pins(prec="mixed", eta=eta)
    try:
        prob = dense_device_problem(C.astype(np.float32), a, b)
        indptr = _zeros(m + 1, torch.int32)
        indices = _zeros(keep, torch.int32)
        data = _zeros(keep)
        assert pins.pins_step_sparsify(h.h, prob.prob, s, dev(F), dev(G), keep, indptr, indices,
                                       data) == 0, h.error()
    finally:
        h.close()
    ip, ix = indptr.cpu().numpy(), indices.cpu().numpy()
    assert ip[-1] == keep
    mask = np.zeros((m, n), dtype=bool)
    for i in range(m):
        mask[i, ix[ip[i]:ip[i + 1]]] = True
    Z = po.log_plan(C, F, G, eta, s)
    slack = 2.0 ** -22 * np.abs(Z).max() + 1e-6
    assert Z[mask].min() >= Z[~mask].max() - slack


# --------------------------------------------------------------------------- #
# CG at the benchmark's sizes and on the fallback path
# --------------------------------------------------------------------------- #
def _stroke_system(gamma, s=40.0, eta=1e-3):
    """A realistic Newton system of a 64 x 64 stroke pair, built with the
    library's own steps (Sinkhorn warm-up, sparsify, marginals) on the FP64
    handle, then brought to the host."""
    import torch
    w = wl.stroke_pair(4, eta=eta, s=64)
    h = pins.Pins(prec="fp64", eta=eta)
    try:
        a, b = dev(w.a), dev(w.b)
        prob = pins.make_problem("grid", a, b, cost_scale=w.cost_scale, grid=w.grid,
                                 on_device=True)
        m, n = w.m, w.n
        F, G = _zeros(m), _zeros(n)
        assert pins.pins_step_sinkhorn(h.h, prob.prob, s, 300, F, G, None) == 0, h.error()
        keep = int(round(gamma * (m + n - 1)))
        indptr, indices, data = _zeros(m + 1, torch.int32), _zeros(keep, torch.int32), _zeros(keep)
        assert pins.pins_step_sparsify(h.h, prob.prob, s, F, G, keep, indptr, indices,
                                       data) == 0, h.error()
        r, c, out = _zeros(m), _zeros(n), _zeros(3)
        assert pins.pins_step_marginals(h.h, prob.prob, s, F, G, r, c, out) == 0, h.error()
    finally:
        h.close()
    r, c = r.cpu().numpy(), c.cpu().numpy()
    rhs = np.concatenate([w.a - r, w.b - c])
    return (m, n, eta, r, c, indptr.cpu().numpy(), indices.cpu().numpy(), data.cpu().numpy(),
            keep, rhs)


def _true_rel(sysd, d):
    from scipy.sparse import csr_matrix, diags, bmat
    m, n, eta, r, c, ip, ix, data, keep, rhs = sysd
    S = csr_matrix((data, ix, ip), shape=(m, n))
    M = bmat([[diags(r), S], [S.T, diags(c)]]).tocsr() / eta
    return np.linalg.norm(M @ d - rhs) / np.linalg.norm(rhs), S


def _run_cg(prec, sysd, rtol, max_iter=20000):
    m, n, eta, r, c, ip, ix, data, keep, rhs = sysd
    d, info = _zeros(m + n), _zeros(2)
    h = pins.Pins(prec=prec, eta=eta)
    try:
        st = pins.pins_step_cg(h.h, m, n, eta, dev(r), dev(c), dev(ip.astype(np.int32)),
                               dev(ix.astype(np.int32)), dev(data), keep, dev(rhs), d, rtol,
                               max_iter, info)
        assert st == 0, h.error()
    finally:
        h.close()
    return d.cpu().numpy(), info.cpu().numpy()


@pytest.mark.parametrize("gamma", [1.0, 2.0, 10.0])
def test_cg_at_8192_unknowns(gamma):
    """16 CTAs x 512 unknowns, the launch the 64 x 64 solves use.  gamma = 10
    gives ~10 000 entries per CTA, too many for shared memory, so the entries
    are read from the global scratch.  Both precisions reach the requested
    residual measured as ||M d - rhs|| (the mixed CG checks it and restarts
    when its recurrences have drifted).  Both follow the oracle's textbook PCG
    in exact arithmetic; FP64 within 2 % of its iteration count, the mixed CG
    (double-float vectors, inner products and step lengths) within 5 %."""
    sysd = _stroke_system(gamma)
    rtol = 1e-6
    it_o = None
    for prec in ("mixed", "fp64"):
        d, info = _run_cg(prec, sysd, rtol)
        assert info[1] <= rtol * 1.0001
        true_rel, S = _true_rel(sysd, d)
        assert true_rel <= 2.0 * rtol + 1e-12
        if it_o is None:
            m, n, eta, r, c, ip, ix, data, keep, rhs = sysd
            csr = po.CSR(m, n, ip.astype(np.int64), ix.astype(np.int64), data)
            _, _, it_o, _ = po.pcg(r, c, csr, eta, rhs[:m], rhs[m:], rtol=rtol, max_iter=20000)
        if prec == "mixed":
            assert abs(int(info[0]) - it_o) <= max(10, it_o // 20)
        else:
            assert abs(int(info[0]) - it_o) <= max(2, it_o // 50)


def test_cg_cooperative_fallback_above_the_cluster_capacity():
    """60 000 unknowns do not fit one cluster's shared memory: both handles run
    the cooperative FP64 PCG, which must meet the residual too."""
    rng = np.random.default_rng(9)
    m = n = 30000
    # a transport-like pattern: each row to its own column and a neighbour, plus
    # random extra entries; values spread over four decades
    rows = np.concatenate([np.arange(m), np.arange(m), rng.integers(0, m, 30000)])
    cols = np.concatenate([np.arange(n), (np.arange(m) + 1) % n, rng.integers(0, n, 30000)])
    lin = np.unique(rows.astype(np.int64) * n + cols)
    rows, cols = lin // n, lin % n
    vals = 10.0 ** rng.uniform(-8, -4, size=lin.size)
    ip = np.zeros(m + 1, dtype=np.int64)
    np.add.at(ip, rows + 1, 1)
    ip = np.cumsum(ip)
    from scipy.sparse import csr_matrix
    S = csr_matrix((vals, cols, ip), shape=(m, n))
    r = np.asarray(S.sum(axis=1)).ravel() * 1.05
    c = np.asarray(S.sum(axis=0)).ravel() * 1.05
    rhs = rng.normal(size=m + n) * 1e-6
    sysd = (m, n, 1e-3, r, c, ip, cols, vals, int(lin.size), rhs)
    for prec in ("mixed", "fp64"):
        d, info = _run_cg(prec, sysd, 1e-6, max_iter=5000)
        assert info[1] <= 1e-6 * 1.0001
        true_rel, _ = _true_rel(sysd, d)
        assert true_rel <= 2e-6


# --------------------------------------------------------------------------- #
# sparsify at full size and on tied keys
# --------------------------------------------------------------------------- #
def _sparsify_fp64(C, a, b, F, G, eta, s, keep):
    import torch
    m, n = C.shape
    h = pins.Pins(prec="fp64", eta=eta)
    try:
        prob = dense_device_problem(C, a, b)
        indptr, indices, data = _zeros(m + 1, torch.int32), _zeros(keep, torch.int32), _zeros(keep)
        st = pins.pins_step_sparsify(h.h, prob.prob, s, dev(F), dev(G), keep, indptr, indices, data)
        err = h.error()
    finally:
        h.close()
    return st, err, indptr.cpu().numpy(), indices.cpu().numpy(), data.cpu().numpy()


def test_sparsify_exact_fp64_at_4096():
    C, a, b, F, G, eta, s = random_state(4096, 4096, 31, eta=1e-2, s=3.0)
    keep = 2 * 4096 - 1
    st, err, ip, ix, data = _sparsify_fp64(C, a, b, F, G, eta, s, keep)
    assert st == 0, err
    S = po.sparsify(C, F, G, eta, s, keep)
    assert np.array_equal(ip, S.indptr) and np.array_equal(ix, S.indices)
    np.testing.assert_allclose(data, S.data, rtol=1e-14)


def test_sparsify_tied_grid_keys():
    """Zero potentials on a grid: keys take one value per squared distance, so
    hundreds of entries tie at the threshold.  16 x 16: the tied entries fit the
    candidate buffer and are ordered by index, exactly as the oracle.  64 x 64:
    16 128 entries tie at distance 1, more than the buffer holds, and the step
    reports its documented error instead of a wrong pattern."""
    for s_grid, ok in ((16, True), (64, False)):
        g = wl.grid_instance(s_grid, 0)
        C = g.dense_cost()
        m = n = g.m
        F, G = np.zeros(m), np.zeros(n)
        keep = m + n - 1
        st, err, ip, ix, data = _sparsify_fp64(C, g.a, g.b, F, G, 1e-2, 1.0, keep)
        if ok:
            assert st == 0, err
            S = po.sparsify(C, F, G, 1e-2, 1.0, keep)
            assert np.array_equal(ip, S.indptr) and np.array_equal(ix, S.indices)
        else:
            assert st == pins.PINS_ERR_CUDA and "tied keys" in err


# --------------------------------------------------------------------------- #
# one-pass selection failure, forced
# --------------------------------------------------------------------------- #
def test_forced_one_pass_failures_redo_the_step_with_the_same_result():
    w = wl.gmm_instance(0, m=300, n=280, eta=1e-2)
    ref = pins.problem_from_workload(w)
    outs = []
    for inject in (0, 6):
        h = pins.Pins(prec="mixed", eta=1e-2, K=4)
        try:
            assert pins.pins_test_inject_faults(h.h, 0, 0, inject) == pins.PINS_OK
            outs.append(h.solve(ref))
        finally:
            h.close()
    a, b = outs
    assert a["newton_iters"] == b["newton_iters"] > 4
    assert a["cost"] == b["cost"]
    assert np.array_equal(a["F"], b["F"]) and np.array_equal(a["G"], b["G"])
