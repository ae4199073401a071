"""The seeded input generators: determinism, valid marginals, the cost
normalisation of each family and the distributions the recipes state."""
import math

import numpy as np
import pytest

from paper_2502_03749_gb300 import workloads as wl


def _valid_marginals(p):
    assert p.a.ndim == 1 and p.b.ndim == 1
    assert np.all(p.a > 0) and np.all(p.b > 0)
    assert abs(p.a.sum() - 1.0) < 1e-12 and abs(p.b.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("make", [
    lambda i: wl.random_assignment(12, i),
    lambda i: wl.small_points(i, m=20, n=30),
    lambda i: wl.gmm_instance(i, m=40, n=50),
    lambda i: wl.grid_instance(9, i),
    lambda i: wl.stroke_pair(i),
    lambda i: wl.serving_request(i, n_min=16, n_max=64),
])
def test_generators_are_seeded_and_draw_valid_marginals(make):
    p, q, r = make(3), make(3), make(4)
    _valid_marginals(p)
    assert np.array_equal(p.a, q.a) and np.array_equal(p.b, q.b)
    assert np.array_equal(p.dense_cost(), q.dense_cost())
    same_shape = p.dense_cost().shape == r.dense_cost().shape and p.a.shape == r.a.shape
    assert not (same_shape and np.array_equal(p.a, r.a) and
                np.array_equal(p.dense_cost(), r.dense_cost()))


def test_max_sq_dist_hull_shortcut_is_exact():
    rng = np.random.default_rng(0)
    for _ in range(5):
        x = rng.normal(size=(50, 2))
        y = rng.normal(size=(70, 2))
        brute = float(np.max(np.sum((x[:, None, :] - y[None, :, :]) ** 2, axis=2)))
        assert wl.max_sq_dist(x, y) == brute


@pytest.mark.parametrize("p", [wl.small_points(0, m=30, n=40, as_dense=False),
                               wl.gmm_instance(1, m=64, n=48, as_dense=False)])
def test_point_costs_are_normalised_to_max_one(p):
    C = p.dense_cost()
    brute = np.sum((p.x[:, None, :] - p.y[None, :, :]) ** 2, axis=2)
    np.testing.assert_allclose(C, p.cost_scale * brute, rtol=1e-15, atol=0)
    assert C.max() == pytest.approx(1.0, rel=1e-15) and C.min() >= 0.0


def test_dense_and_point_forms_agree():
    pts = wl.gmm_instance(2, m=33, n=35, as_dense=False)
    den = wl.gmm_instance(2, m=33, n=35, as_dense=True)
    np.testing.assert_allclose(den.C, pts.dense_cost(), rtol=1e-15, atol=1e-18)


def test_grid_cost_definition_and_normalisation():
    s = 7
    p = wl.grid_instance(s, 0)
    C = p.dense_cost()
    assert C.shape == (s * s, s * s) and p.m == p.n == s * s
    for i, j in [(0, 48), (3, 3), (10, 37), (48, 0)]:
        i1, i2, j1, j2 = i // s, i % s, j // s, j % s
        assert C[i, j] == p.cost_scale * ((i1 - j1) ** 2 + (i2 - j2) ** 2)
    assert C.max() == 1.0 and np.array_equal(C, C.T)


def test_stroke_pairs_use_the_stated_grids():
    sizes = set()
    for i in range(40):
        p = wl.stroke_pair(i)
        s = p.grid[0]
        assert p.grid == (s, s) and s in wl.STROKE_GRIDS and p.m == s * s
        _valid_marginals(p)
        sizes.add(s)
    assert sizes == set(wl.STROKE_GRIDS)


def test_serving_sizes_are_log_uniform_in_range():
    ns = np.array([wl.serving_request(i, n_min=4, n_max=64).n for i in range(400)])
    assert ns.min() >= 4 and ns.max() <= 64
    # log-uniform on [ln 4, ln 64]: the median is near the geometric mean 16 and
    # a quarter of the draws fall below 8 (= 4 * 16^(1/4))
    assert 13 <= np.median(ns) <= 20
    assert 0.17 <= np.mean(ns < 8) <= 0.33


def test_poisson_arrivals_have_the_stated_rate():
    t = wl.poisson_arrivals(100.0, 4000, 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 0.01) < 0.01 * 4 / math.sqrt(4000) * 1.5
