"""Serving error paths, with every fault made on the host (no GPU fault):
queue overflow, a request above the memory budget, an injected allocation
failure and an injected kernel error word, each returning its status while the
worker pool keeps serving; and memory admission that counts every arena the
pool holds, so a small budget with mixed request sizes never runs out."""
import time

import numpy as np
import pytest

from paper_2502_03749_gb300 import pins, workloads as wl

pytestmark = pytest.mark.gpu


def _small(i, s=12):
    g = wl.grid_instance(s, i, eta=1e-2)
    return pins.problem_from_workload(g)


def _wait_all(h, tickets):
    return [h.wait(t) for t in tickets]


def test_queue_overflow_returns_queue_full_and_the_pool_keeps_serving():
    h = pins.Pins(eta=1e-2, K=20, max_inflight=1, queue_capacity=2)
    try:
        slow = pins.problem_from_workload(wl.stroke_pair(3, eta=1e-3, s=48))
        tickets, full = [h.submit(slow)], 0
        smalls = [_small(i) for i in range(6)]      # keep the arrays alive
        for ref in smalls:
            st, t = pins.pins_submit(h.h, ref.prob)
            if st == pins.PINS_ERR_QUEUE_FULL:
                full += 1
            else:
                assert st == pins.PINS_OK
                tickets.append(t)
        assert full >= 3
        assert "queue full" in h.error()
        for d in _wait_all(h, tickets):
            assert d["status"] in (pins.PINS_OK, pins.PINS_ERR_NOT_CONVERGED)
        d = h.wait(h.submit(_small(9)))
        assert d["status"] in (pins.PINS_OK, pins.PINS_ERR_NOT_CONVERGED)
    finally:
        h.close()


def _held_after_one(prob, **cfg):
    h = pins.Pins(max_inflight=1, **cfg)
    try:
        h.wait(h.submit(prob))
        return pins.pins_serving_held_bytes(h.h)[0]
    finally:
        h.close()


def test_request_above_the_budget_is_rejected_at_submit():
    small = _held_after_one(_small(0, s=6), eta=1e-2, K=5)
    h = pins.Pins(eta=1e-2, K=5, max_inflight=2, device_mem_budget=int(1.5 * small))
    try:
        big = pins.problem_from_workload(wl.grid_instance(48, 0))
        st, _ = pins.pins_submit(h.h, big.prob)
        assert st == pins.PINS_ERR_OOM
        assert "budget" in h.error()
        d = h.wait(h.submit(_small(0, s=6)))
        assert d["status"] in (pins.PINS_OK, pins.PINS_ERR_NOT_CONVERGED)
    finally:
        h.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_injected_allocation_failure_and_kernel_error(prec):
    """The next allocation fails (PINS_ERR_OOM), then the next kernel error word
    is set (PINS_ERR_CUDA); requests after each succeed on the same pool, and a
    blocking solve on the handle behaves the same."""
    h = pins.Pins(eta=1e-2, K=3, prec=prec, max_inflight=1)
    try:
        assert pins.pins_test_inject_faults(h.h, 1, 0) == pins.PINS_OK
        d = h.wait(h.submit(_small(1, s=10)))
        assert d["status"] == pins.PINS_ERR_OOM and "injected" in h.error()
        d = h.wait(h.submit(_small(2, s=10)))
        assert d["status"] in (pins.PINS_OK, pins.PINS_ERR_NOT_CONVERGED)
        assert pins.pins_test_inject_faults(h.h, 0, 1) == pins.PINS_OK
        d = h.wait(h.submit(_small(3, s=10)))
        assert d["status"] == pins.PINS_ERR_CUDA and "injected" in h.error()
        d = h.wait(h.submit(_small(4, s=10)))
        assert d["status"] in (pins.PINS_OK, pins.PINS_ERR_NOT_CONVERGED)
        assert pins.pins_test_inject_faults(h.h, 0, 1) == pins.PINS_OK
        res = pins.pins_result()
        ref = _small(5, s=10)
        assert pins.pins_solve(h.h, ref.prob, res) == pins.PINS_ERR_CUDA
        assert pins.pins_solve(h.h, ref.prob, res) in (pins.PINS_OK, pins.PINS_ERR_NOT_CONVERGED)
        assert pins.pins_test_inject_faults(h.h, -1, 0) == pins.PINS_ERR_INVALID_ARG
    finally:
        h.close()


def test_admission_counts_every_arena_the_pool_holds():
    """Budget for about two large requests; a stream alternating large and small
    requests on four workers: no request fails for memory, and the pool's arenas
    never exceed the budget while several run."""
    sizes = [48, 12, 40, 10, 48, 16, 44, 12, 48, 10]
    probs = [pins.problem_from_workload(wl.grid_instance(s, i, eta=1e-2))
             for i, s in enumerate(sizes)]
    big = _held_after_one(probs[0], eta=1e-2, K=4)
    budget = int(2.2 * big)
    h = pins.Pins(eta=1e-2, K=4, max_inflight=4, device_mem_budget=budget)
    try:
        tickets = [h.submit(p) for p in probs]
        peak = 0
        pending = set(tickets)
        while pending:
            held, b = pins.pins_serving_held_bytes(h.h)
            assert b == budget
            peak = max(peak, held)
            for t in list(pending):
                d = h.poll(t)
                if d is not None:
                    assert d["status"] in (pins.PINS_OK, pins.PINS_ERR_NOT_CONVERGED), h.error()
                    pending.discard(t)
            time.sleep(0.001)
        assert peak <= budget
    finally:
        h.close()
