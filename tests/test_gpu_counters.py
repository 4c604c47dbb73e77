"""Interaction counters of the walks (sph_profile_counters), checked where
they have an exact value: the partner walk finds exactly the partners of the
lists (the sum of the partner counts) and tests at least as many candidates;
the Barnes-Hut walk at opening angle 0 opens every node, so it uses no node as
a pseudo-particle and sums every pair directly, n (n - 1) terms; at 0.5 it
uses nodes and sums fewer terms.  Nothing is counted while profiling is off."""
from dataclasses import replace

import numpy as np
import pytest

from paper_1604_03290_gb300 import workloads as wl
from parity_util import flawed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_03290_gb300 import sph
    return sph


def test_partner_walk_counts_its_partners(S):
    ps = flawed(wl.measurement_1m(seed=3, n_side=16))
    ctx = S.Context(3, ps.n, max_neighbours=160)
    ctx.profile(True)
    off, idx = S.neighbours(ctx, S.DeviceState(ps), 16, 21)
    c = ctx.profile_counters()
    assert c["walk_partners"] == int(off[-1].item())
    assert c["walk_tests"] >= c["walk_partners"] > 0
    assert c["grav_nodes"] == c["grav_terms"] == 0
    ctx.profile(False)
    S.neighbours(ctx, S.DeviceState(ps), 16, 21)
    ctx.profile(True)
    assert all(v == 0 for v in ctx.profile_counters().values())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gravity_counts_at_opening_angles_0_and_half(S, prec):
    cl = wl.cloud_collapse(seed=3, n=3000)
    ctx = S.Context(3, cl.n, max_neighbours=160)
    ctx.profile(True)
    S.gravity(ctx, S.DeviceState(cl), replace(cl.params, precision=prec, theta=0.0))
    c0 = ctx.profile_counters()
    assert c0["grav_nodes"] == 0
    assert c0["grav_terms"] == cl.n * (cl.n - 1)
    S.gravity(ctx, S.DeviceState(cl), replace(cl.params, precision=prec, theta=0.5))
    c5 = ctx.profile_counters()
    assert c5["grav_nodes"] > 0 and c5["grav_terms"] < c0["grav_terms"]
    assert c5["grav_visits"] > 0
