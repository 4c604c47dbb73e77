"""Seeded input generators: shapes, counts and the flaw distribution of Sect. 3.2."""
import math

import numpy as np
import pytest

from paper_1604_03290_gb300 import workloads as wl


def test_weibull_flaws_cover_every_particle():
    rng = np.random.default_rng(0)
    n = 20000
    k, m, V = 5e34, 8.5, 3.0
    off, eps = wl.weibull_flaws(rng, n, V, k, m)
    cnt = np.diff(off)
    assert cnt.min() >= 1
    # about N ln N flaws in total (coupon collector: N (ln N + 0.577))
    assert abs(off[-1] / (n * (math.log(n) + 0.5772)) - 1) < 0.1
    for a in range(0, n, 997):
        e = eps[off[a]:off[a + 1]]
        assert np.all(np.diff(e) >= 0)
    # the thresholds are (j / (k V))^(1/m) for j = 1..N_flaw
    allj = np.sort(eps.astype(np.float64))
    ref = (np.arange(1, off[-1] + 1) / (k * V)) ** (1 / m)
    np.testing.assert_allclose(allj, ref, rtol=1e-6)


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
    np.testing.assert_array_equal(a.flaw_eps, b.flaw_eps)
    np.testing.assert_array_equal(a.S, b.S)
