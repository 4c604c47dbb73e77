"""Pins of the oracle's time-step limits (Sect. 3.4.1; readings: the
acceleration limit c_a sqrt(h/|a|), the quantity limits c_q (|q| + floor)/|dq/dt|
with per-field floors).  Each limit is switched on alone through synthetic
derivatives and must give its closed form; then the minimum over limits and
particles, the instances' independence, the density limit skipped with the
kernel-sum density, damage limited only while it grows, dt_max and dt_fixed."""
from dataclasses import replace

import numpy as np
import pytest

from paper_1604_03290_gb300 import workloads as wl


def _state(n=40, dim=3, seed=0, inst_off=None):
    rng = np.random.default_rng(seed)
    ps = wl.lattice_block(seed=seed, nx=n, ny=1, nz=1, dim=dim, jitter=0.1)
    ps.h = rng.uniform(0.5, 2.0, ps.n)
    ps.rho = rng.uniform(0.5, 2.0, ps.n)
    ps.u = rng.uniform(-3.0, 3.0, ps.n)
    ps.S = rng.normal(0.0, 2.0, (6 if dim == 3 else 3, ps.n))
    ps.dmg = rng.uniform(0.0, 0.9, ps.n)
    ps.inst_off = inst_off
    return ps


def _zero(ps):
    n, dim = ps.n, ps.dim
    return {"dv": np.zeros((dim, n)), "drho": np.zeros(n), "du": np.zeros(n), "cs": np.zeros(n),
            "dS": np.zeros((6 if dim == 3 else 3, n)), "ddmg": np.zeros(n)}


P = wl.Params(dim=3, c_courant=0.7, c_accel=0.2, c_quantity=0.7, u_floor=0.5, S_floor=0.25, dmg_floor=0.01)


def test_nothing_limits_gives_dt_max(orc):
    ps = _state()
    assert orc.timestep(ps, ps.materials, replace(P, dt_max=3.5), _zero(ps))[0] == 3.5


def test_courant_limit(orc):
    ps = _state(seed=1)
    d = _zero(ps)
    d["cs"] = np.random.default_rng(2).uniform(0.5, 3.0, ps.n)
    np.testing.assert_allclose(orc.timestep(ps, ps.materials, P, d)[0], (0.7 * ps.h / d["cs"]).min(), rtol=1e-15)


def test_acceleration_limit(orc):
    ps = _state(seed=3)
    d = _zero(ps)
    d["dv"] = np.random.default_rng(4).normal(0.0, 5.0, d["dv"].shape)
    amag = np.sqrt((d["dv"] ** 2).sum(0))
    np.testing.assert_allclose(orc.timestep(ps, ps.materials, P, d)[0], (0.2 * np.sqrt(ps.h / amag)).min(),
                               rtol=1e-15)


@pytest.mark.parametrize("field,floor", [("rho", 0.0), ("u", 0.5)])
def test_density_and_energy_limits(orc, field, floor):
    ps = _state(seed=5)
    d = _zero(ps)
    rate = np.random.default_rng(6).normal(0.0, 4.0, ps.n)
    d["d" + field] = rate
    q = getattr(ps, field)
    want = (0.7 * (np.abs(q) + floor) / np.abs(rate)).min()
    np.testing.assert_allclose(orc.timestep(ps, ps.materials, P, d)[0], want, rtol=1e-15)
    if field == "rho":  # the kernel-sum density is not integrated, so it does not limit
        assert orc.timestep(ps, ps.materials, replace(P, density_sum=True), d)[0] == P.dt_max


def test_stress_limit_per_component(orc):
    ps = _state(seed=7)
    d = _zero(ps)
    rng = np.random.default_rng(8)
    d["dS"] = rng.normal(0.0, 3.0, d["dS"].shape)
    d["dS"][:, ::3] = 0.0  # zero rates do not limit
    with np.errstate(divide="ignore"):
        lim = np.where(d["dS"] != 0.0, 0.7 * (np.abs(ps.S) + 0.25) / np.abs(d["dS"]), np.inf)
    np.testing.assert_allclose(orc.timestep(ps, ps.materials, P, d)[0], lim.min(), rtol=1e-15)


def test_damage_limits_only_while_growing(orc):
    ps = _state(seed=9)
    d = _zero(ps)
    rate = np.random.default_rng(10).normal(0.0, 2.0, ps.n)
    d["ddmg"] = rate
    grow = rate > 0
    want = (0.7 * (np.abs(ps.dmg[grow]) + 0.01) / rate[grow]).min()
    np.testing.assert_allclose(orc.timestep(ps, ps.materials, P, d)[0], want, rtol=1e-15)
    d["ddmg"] = -np.abs(rate)
    assert orc.timestep(ps, ps.materials, P, d)[0] == P.dt_max


def test_minimum_over_limits_and_instances(orc):
    off = np.array([0, 10, 25, 40], np.int64)
    ps = _state(seed=11, inst_off=off)
    rng = np.random.default_rng(12)
    d = _zero(ps)
    d["cs"] = rng.uniform(0.5, 3.0, ps.n)
    d["dv"] = rng.normal(0.0, 50.0, d["dv"].shape)
    d["du"] = rng.normal(0.0, 30.0, ps.n)
    lim = np.minimum.reduce([0.7 * ps.h / d["cs"], 0.2 * np.sqrt(ps.h / np.sqrt((d["dv"] ** 2).sum(0))),
                             0.7 * (np.abs(ps.u) + 0.5) / np.abs(d["du"])])
    dt = orc.timestep(ps, ps.materials, P, d)
    np.testing.assert_allclose(dt, [lim[off[i]:off[i + 1]].min() for i in range(3)], rtol=1e-15)
    # an instance's step does not see the other instances: make instance 0 stiff
    d["cs"][:10] *= 1e3
    dt2 = orc.timestep(ps, ps.materials, P, d)
    assert dt2[0] < dt[0] and dt2[1] == dt[1] and dt2[2] == dt[2]
    # a fixed step overrides every limit
    np.testing.assert_array_equal(orc.timestep(ps, ps.materials, replace(P, dt_fixed=0.125), d), [0.125] * 3)
