"""Seeded input generators: shapes, counts, seeds (the flaws of Sect. 3.2 are drawn by the
library's and the oracle's generators from the workloads' flaw seeds)."""
import math

import numpy as np
import pytest

from paper_1604_03290_gb300 import workloads as wl


def test_workload_shapes():
    r = wl.rings_2d()
    assert r.dim == 2 and 4300 < r.n < 4500
    assert np.all(r.v[0, r.x[0] < 0] > 0) and np.all(r.v[0, r.x[0] > 0] < 0)
    a = wl.al_impact(n_side=64)
    assert 1000 < a.n - 64 ** 3 < 1200  # ~1,100 sphere particles
    c = wl.cloud_collapse(n=20000)
    assert c.m.sum() == pytest.approx(wl.M_SUN, rel=1e-12)
    assert abs(c.n / 20000 - 1) < 0.05
    b = wl.batched_impacts(ninst=8, with_flaws=False)
    assert b.ninst == 8 and b.inst_off[-1] == b.n
    sizes = np.diff(b.inst_off)
    assert sizes.min() >= 2000 * 0.8 and sizes.max() <= 50000 * 1.3


def test_generators_are_seeded():
    a = wl.measurement_1m(n_side=10)
    b = wl.measurement_1m(n_side=10)
    np.testing.assert_array_equal(a.x, b.x)
    assert a.flaw_seed == b.flaw_seed is not None and a.flaw_off is None
    np.testing.assert_array_equal(a.S, b.S)
