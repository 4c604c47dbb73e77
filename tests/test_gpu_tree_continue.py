"""A window of steps on one tree spanning several sph_step calls
(params.tree_reuse with tree_continue): one-step calls that continue the
window, with the state copied to the host and back between them, must give
the states of one call over all the steps bit for bit; a continuation after
another call on the context, after a change of the state, or with other
settings is refused with SPH_ERR_INVALID before any work."""
from dataclasses import replace

import numpy as np
import pytest

from paper_1604_03290_gb300 import workloads as wl
from parity_util import flawed

pytestmark = pytest.mark.gpu

FIELDS = ("x", "v", "rho", "u", "S", "dmg", "h", "id")


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_03290_gb300 import sph
    return sph


def _case():
    ps = flawed(wl.measurement_1m(seed=41, n_side=20))
    ps.params = replace(ps.params, tree_reuse=4)
    return ps


def _ctx(S, ps):
    return S.Context(3, ps.n, max_neighbours=160, leaf_size=ps.params.leaf_size)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_continued_calls_equal_one_call(S, prec):
    ps = _case()
    prm = replace(ps.params, precision=prec)
    nsteps = 7  # a build, 3 continued steps, a build, 2 continued steps
    ctx = _ctx(S, ps)
    ds = S.DeviceState(ps)
    dt_one = S.step(ctx, ds, ps.materials, prm, nsteps).cpu().numpy()
    one = ds.to_numpy()
    ctx2 = _ctx(S, ps)
    ds2 = S.DeviceState(ps)
    ctx2.profile(True)
    for i in range(nsteps):
        dt = S.step(ctx2, ds2, ps.materials, prm, 1, cont=i > 0).cpu().numpy()
        # out to the host and back into the same device buffers
        for k in FIELDS:
            t = getattr(ds2, k)
            if t is not None:
                t.copy_(t.cpu())
    ph = ctx2.profile_read()
    many = ds2.to_numpy()
    for k in FIELDS:
        if one.get(k) is not None:
            np.testing.assert_array_equal(many[k], one[k], err_msg=k)
    np.testing.assert_array_equal(dt, dt_one)
    assert ph["reorder"][1] == 2  # trees built at steps 0 and 4 only


def test_continuation_refused_after_other_calls_or_changes(S):
    ps = _case()
    prm = replace(ps.params, precision="mixed")
    ctx = _ctx(S, ps)
    ds = S.DeviceState(ps)
    S.step(ctx, ds, ps.materials, prm, 1)
    # another call on the context in between
    S.rhs(ctx, S.DeviceState(ps), ps.materials, prm)
    with pytest.raises(S.SphError) as e:
        S.step(ctx, ds, ps.materials, prm, 1, cont=True)
    assert e.value.status == S.SPH_ERR_INVALID and "previous call" in str(e.value)
    # a position one ulp away from the returned one
    S.step(ctx, ds, ps.materials, prm, 1)
    import torch
    ds.x[0, 5] = torch.nextafter(ds.x[0, 5], torch.tensor(np.inf, dtype=torch.float64, device=ds.x.device))
    with pytest.raises(S.SphError) as e:
        S.step(ctx, ds, ps.materials, prm, 1, cont=True)
    assert e.value.status == S.SPH_ERR_INVALID and "differ" in str(e.value)
    # other settings than the window's
    S.step(ctx, ds, ps.materials, prm, 1)
    with pytest.raises(S.SphError) as e:
        S.step(ctx, ds, ps.materials, replace(prm, tree_reuse=2), 1, cont=True)
    assert e.value.status == S.SPH_ERR_INVALID
    # and the context still steps afterwards, continuing a fresh window
    S.step(ctx, ds, ps.materials, prm, 1)
    S.step(ctx, ds, ps.materials, prm, 1, cont=True)
