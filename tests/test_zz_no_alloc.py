"""The allocation-free marginal pass, pins_marginals_noalloc.

It exists for callers that cannot allocate device memory (a framework that owns
all device memory through its own pool, a real-time loop that must not enter the
driver's allocator): its scratch is a static device array set up on the first
call.  Here it is checked against the handle-based pins_step_marginals on calls
in a row -- different sizes back to back, then a repeat -- so a result left in
the shared scratch by one call cannot leak into the next.  This file is named to
run last; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from oracle import pins_oracle as po
from paper_2502_03749_gb300 import pins, workloads as wl

from gpu_util import dense_device_problem, dev, random_state

pytestmark = pytest.mark.gpu

MAX_DIM = 4096   # PINS_NOALLOC_MAX_DIM in include/pins.h


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_matches_handle_entry_point_on_calls_in_a_row(prec):
    import torch
    mixed = prec == "mixed"
    h = pins.Pins(prec=prec, eta=0.05)
    try:
        for call, (m, n) in enumerate([(200, 333), (70, 150), (200, 333)]):
            C, a, b, F, G, eta, s = random_state(m, n, 1000 + (call % 2))
            prob = dense_device_problem(C.astype(np.float32) if mixed else C, a, b)
            Fd, Gd = dev(F), dev(G)
            r0 = torch.zeros(m, dtype=torch.float64, device="cuda")
            c0 = torch.zeros(n, dtype=torch.float64, device="cuda")
            o0 = torch.zeros(3, dtype=torch.float64, device="cuda")
            st = pins.pins_step_marginals(h.h, prob.prob, s, Fd, Gd, r0, c0, o0)
            assert st == pins.PINS_OK, h.error()
            r1 = torch.full((m,), -1.0, dtype=torch.float64, device="cuda")
            c1 = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
            o1 = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
            st = pins.pins_marginals_noalloc(prob.prob, eta,
                                             pins.PINS_PREC_MIXED if mixed else pins.PINS_PREC_FP64,
                                             s, Fd, Gd, r1, c1, o1, None)
            assert st == pins.PINS_OK
            torch.cuda.synchronize()
            tol = 1e-10 if mixed else 1e-12
            np.testing.assert_allclose(r1.cpu().numpy(), r0.cpu().numpy(), rtol=tol)
            np.testing.assert_allclose(c1.cpu().numpy(), c0.cpu().numpy(), rtol=tol)
            np.testing.assert_allclose(o1.cpu().numpy(), o0.cpu().numpy(), rtol=tol, atol=1e-15)
    finally:
        h.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    m, n = MAX_DIM + 1, 2
    a = np.full(m, 1.0 / m)
    b = np.full(n, 0.5)
    C = np.zeros((m, n))
    prob = dense_device_problem(C, a, b)
    F = torch.zeros(m, dtype=torch.float64, device="cuda")
    G = torch.zeros(n, dtype=torch.float64, device="cuda")
    r = torch.zeros(m, dtype=torch.float64, device="cuda")
    c = torch.zeros(n, dtype=torch.float64, device="cuda")
    o = torch.zeros(3, dtype=torch.float64, device="cuda")
    st = pins.pins_marginals_noalloc(prob.prob, 0.05, pins.PINS_PREC_FP64, 1.0, F, G, r, c, o, None)
    assert st == pins.PINS_ERR_INVALID_ARG


def _noalloc(prob, eta, mixed, s, F, G, m, n):
    import torch
    r = torch.full((m,), -1.0, dtype=torch.float64, device="cuda")
    c = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    o = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
    st = pins.pins_marginals_noalloc(prob.prob, eta,
                                     pins.PINS_PREC_MIXED if mixed else pins.PINS_PREC_FP64,
                                     s, dev(F), dev(G), r, c, o, None)
    assert st == pins.PINS_OK
    torch.cuda.synchronize()
    return r.cpu().numpy(), c.cpu().numpy(), o.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["points2", "points3", "grid"])
def test_noalloc_streamed_cost_kinds_match_handle_entry_point(prec, kind):
    """Point clouds (d = 2 and 3; the mixed path converts their coordinates into
    the static scratch) and grids (cost from indices), two calls in a row."""
    import torch
    mixed = prec == "mixed"
    eta, s = 0.05, 2.0
    h = pins.Pins(prec=prec, eta=eta)
    try:
        for call in range(2):
            rng = np.random.default_rng(77 + call)
            if kind == "grid":
                g = wl.grid_instance(13 + 3 * call, call)
                m = n = g.m
                prob = pins.make_problem("grid", dev(g.a), dev(g.b), cost_scale=g.cost_scale,
                                         grid=g.grid, on_device=True)
            else:
                d = 2 if kind == "points2" else 3
                m, n = 150 + 37 * call, 211 - 50 * call
                x, y = rng.uniform(0, 1, (m, d)), rng.uniform(0, 1, (n, d))
                a = rng.uniform(0.5, 1.5, m); a /= a.sum()
                b = rng.uniform(0.5, 1.5, n); b /= b.sum()
                prob = pins.make_problem("points", dev(a), dev(b), x=dev(x), y=dev(y),
                                         cost_scale=1.0 / d, on_device=True)
            F = rng.normal(size=m) * 0.02 - 0.05
            G = rng.normal(size=n) * 0.02
            r0 = torch.zeros(m, dtype=torch.float64, device="cuda")
            c0 = torch.zeros(n, dtype=torch.float64, device="cuda")
            o0 = torch.zeros(3, dtype=torch.float64, device="cuda")
            st = pins.pins_step_marginals(h.h, prob.prob, s, dev(F), dev(G), r0, c0, o0)
            assert st == pins.PINS_OK, h.error()
            r1, c1, o1 = _noalloc(prob, eta, mixed, s, F, G, m, n)
            tol = 1e-10 if mixed else 1e-12
            np.testing.assert_allclose(r1, r0.cpu().numpy(), rtol=tol)
            np.testing.assert_allclose(c1, c0.cpu().numpy(), rtol=tol)
            np.testing.assert_allclose(o1, o0.cpu().numpy(), rtol=tol, atol=1e-15)
    finally:
        h.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_at_its_maximum_size_against_the_oracle(prec):
    """The documented maximum, 4096 x 4096, then 4096 x 1 and a small call right
    after: every row and column sum against the oracle (FP64 1e-12, mixed 1e-10
    relative), so the scratch layout holds the largest launch and nothing of the
    large call carries over."""
    mixed = prec == "mixed"
    for (m, n) in [(MAX_DIM, MAX_DIM), (MAX_DIM, 1), (37, 53)]:
        rng = np.random.default_rng(m + 3 * n)
        C = rng.uniform(0, 1, size=(m, n))
        if mixed:
            C = C.astype(np.float32).astype(np.float64)
        a = rng.uniform(0.5, 1.5, m); a /= a.sum()
        b = rng.uniform(0.5, 1.5, n); b /= b.sum()
        eta, s = 0.05, 2.0
        F, G = np.zeros(m), np.zeros(n)
        F, _ = po.sinkhorn_row_step(C, a, F, G, eta, s)
        G = po.sinkhorn_col_step(C, b, F, G, eta, s)
        prob = dense_device_problem(C.astype(np.float32) if mixed else C, a, b)
        r1, c1, o1 = _noalloc(prob, eta, mixed, s, F, G, m, n)
        _, _, r0, c0 = po.gradient(C, a, b, F, G, eta, s)
        tol = 1e-10 if mixed else 1e-12
        np.testing.assert_allclose(r1, r0, rtol=tol)
        np.testing.assert_allclose(c1, c0, rtol=tol)
        # the l1 residual sums m + n differences of nearly equal numbers: each
        # row sum carries the path's relative rounding (1e-10 mixed)
        assert o1[0] == pytest.approx(po.residual_l1(a, b, r0, c0), rel=1e-8,
                                      abs=1e-11 if mixed else 1e-14)
        assert o1[1] == pytest.approx(r0.sum(), rel=tol)
