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

from paper_2502_03749_gb300 import pins

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
