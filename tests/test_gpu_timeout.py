"""Device loops that run out of iterations report SPH_ERR_TIMEOUT and leave
the context usable.

Every walk and union-find loop in the library is bounded; reaching the bound
stops the loop, sets the device error word and the call returns
SPH_ERR_TIMEOUT.  The test lowers the bound through sph_tuning.iter_cap to a
value the inputs are sure to exceed (a walk of at most two nodes, one pointer
step per find), so the loops stop early without any fault, then restores the
default bound and requires the results of an untouched context bit for bit.
"""
from dataclasses import replace

import numpy as np
import pytest

from paper_1604_03290_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_03290_gb300 import sph
    return sph


def _expect_timeout(S, fn):
    with pytest.raises(S.SphError) as e:
        fn()
    assert e.value.status == S.SPH_ERR_TIMEOUT, str(e.value)
    assert "iteration limit" in str(e.value)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_partner_walk_timeout_then_recovers(S, prec):
    ps = wl.al_impact(n_side=16)
    P = replace(ps.params, precision=prec)
    ref = S.rhs(S.Context(3, ps.n, max_neighbours=128), S.DeviceState(ps), ps.materials, P)
    ctx = S.Context(3, ps.n, max_neighbours=128)
    ctx.set_tuning(iter_cap=2)
    _expect_timeout(S, lambda: S.rhs(ctx, S.DeviceState(ps), ps.materials, P))
    ctx.set_tuning(iter_cap=0)
    out = S.rhs(ctx, S.DeviceState(ps), ps.materials, P)
    for f in ("dv", "du", "drho", "dS"):
        np.testing.assert_array_equal(out[f].cpu().numpy(), ref[f].cpu().numpy(), err_msg=f)


def test_gravity_walk_timeout_then_recovers(S):
    cl = wl.cloud_collapse(seed=3, n=4000)
    P = replace(cl.params, precision="mixed")
    ref = S.gravity(S.Context(3, cl.n, max_neighbours=160), S.DeviceState(cl), P).cpu().numpy()
    ctx = S.Context(3, cl.n, max_neighbours=160)
    ctx.set_tuning(iter_cap=2)
    _expect_timeout(S, lambda: S.gravity(ctx, S.DeviceState(cl), P))
    ctx.set_tuning(iter_cap=0)
    np.testing.assert_array_equal(S.gravity(ctx, S.DeviceState(cl), P).cpu().numpy(), ref)


def test_fragment_union_timeout_then_recovers(S):
    ps = wl.al_impact(n_side=16)
    ps.dmg = np.zeros(ps.n)
    ref = [t.cpu().numpy() for t in S.fragments(S.Context(3, ps.n, max_neighbours=128), S.DeviceState(ps))]
    ctx = S.Context(3, ps.n, max_neighbours=128)
    # one node per walk and one pointer step per find: the finder's partner
    # walk and its union both run out
    ctx.set_tuning(iter_cap=1)
    _expect_timeout(S, lambda: S.fragments(ctx, S.DeviceState(ps)))
    ctx.set_tuning(iter_cap=0)
    got = [t.cpu().numpy() for t in S.fragments(ctx, S.DeviceState(ps))]
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g, r)
