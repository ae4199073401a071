"""Argument marshalling of the Python binding, checked without a GPU: the
pins_problem a caller builds points at contiguous arrays of the C ABI's types,
in the layout the header states, and keeps them alive."""
import ctypes as ct

import numpy as np
import pytest

from paper_2502_03749_gb300 import pins, workloads as wl


def _read(ptr, dtype, count):
    ctype = {np.float64: ct.c_double, np.float32: ct.c_float}[dtype]
    return np.ctypeslib.as_array(ct.cast(ptr, ct.POINTER(ctype)), shape=(count,)).copy()


def test_dense_fp64_problem_points_at_row_major_copies():
    w = wl.small_points(0, m=5, n=7)
    C = np.asfortranarray(w.C)                       # not C-contiguous on purpose
    ref = pins.make_problem("dense", w.a, w.b, C=C)
    p = ref.prob
    assert (p.m, p.n, p.kind, p.on_device) == (5, 7, pins.PINS_COST_DENSE_F64, 0)
    np.testing.assert_array_equal(_read(p.C, np.float64, 35), w.C.ravel(order="C"))
    np.testing.assert_array_equal(_read(p.a, np.float64, 5), w.a)
    np.testing.assert_array_equal(_read(p.b, np.float64, 7), w.b)


def test_dense_fp32_problem_keeps_fp32():
    w = wl.small_points(1, m=4, n=3)
    C32 = w.C.astype(np.float32)
    p = pins.make_problem("dense", w.a, w.b, C=C32).prob
    assert p.kind == pins.PINS_COST_DENSE_F32
    np.testing.assert_array_equal(_read(p.C, np.float32, 12), C32.ravel())


def test_points_and_grid_problems():
    w = wl.gmm_instance(0, m=6, n=9, as_dense=False)
    p = pins.problem_from_workload(w).prob
    assert p.kind == pins.PINS_COST_POINTS_SQEUCLID and p.d == 2
    assert p.cost_scale == w.cost_scale
    np.testing.assert_array_equal(_read(p.x, np.float64, 12), w.x.ravel())
    np.testing.assert_array_equal(_read(p.y, np.float64, 18), w.y.ravel())
    g = wl.grid_instance(5, 0)
    pg = pins.problem_from_workload(g).prob
    assert pg.kind == pins.PINS_COST_GRID_SQEUCLID and (pg.grid_s1, pg.grid_s2) == (5, 5)
    assert pg.m == pg.n == 25 and not pg.C and not pg.x


def test_problem_from_workload_can_materialise_the_cost():
    w = wl.gmm_instance(3, m=4, n=5, as_dense=False)
    p = pins.problem_from_workload(w, as_kind="dense").prob
    assert p.kind == pins.PINS_COST_DENSE_F64
    np.testing.assert_array_equal(_read(p.C, np.float64, 20), w.dense_cost().ravel())


def test_unknown_kind_is_rejected():
    with pytest.raises(ValueError):
        pins.make_problem("sparse", np.ones(2) / 2, np.ones(2) / 2)


def test_config_fields_are_set_by_name_and_unknown_names_raise(monkeypatch):
    # pins_create is replaced: only the field marshalling of Pins(...) is checked
    seen = {}
    monkeypatch.setattr(pins, "pins_config_default", lambda: pins.pins_config())
    monkeypatch.setattr(pins, "pins_create", lambda c: seen.setdefault("cfg", c) and None)
    h = pins.Pins(prec="mixed", eta=0.05, K=7, T2=0, sparsify_one_pass=0)
    c = seen["cfg"]
    assert c.prec == pins.PINS_PREC_MIXED and c.eta == 0.05 and c.K == 7 and c.T2 == 0
    assert c.sparsify_one_pass == 0
    h.h = None
    with pytest.raises(KeyError):
        pins.Pins(no_such_field=1)
