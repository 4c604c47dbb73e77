"""Partners of the later evaluations of a step refined from the step's first
walk (its lists plus the candidates within (1 + 1/64) h_ab) against a tree
walk at every evaluation: the states and time steps must be bit-identical,
because the refined lists are the same sets in the same ascending order.
Covered: an impact whose predictor moves particles by ~1e-4 h (the lists are
refined), the same impact with a fixed step that moves the projectile by half
its support radius (the bound fails and the walk runs), a lattice whose
shells hold more candidates than their slots (the walk runs), batched instances,
2D rings with XSPH and artificial stress, a self-gravitating pair stepping
with a reused tree, the impact on a tree reused for 3 steps (every evaluation
after a build refines from the build step's walk) and for 6 steps with a
longer step (the bound fails within the window), and the embedded
Runge-Kutta step; FP64 and mixed."""
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


def _impact():
    return flawed(wl.measurement_1m(seed=31, n_side=18))


def _impact_fast():
    ps = flawed(wl.measurement_1m(seed=33, n_side=14))
    hp = ps.h[ps.v[2] < -1000.0].min()
    ps.params = replace(ps.params, dt_fixed=2 * 0.5 * hp / 7000.0)
    return ps


def _batch():
    ps = flawed(wl.batched_impacts(seed=5, ninst=4, nmin=400, nmax=1500))
    ps.params = replace(ps.params, max_depth=19)
    return ps


def _rings():
    ps = wl.rings_2d(artificial_stress=True)
    ps.params = replace(ps.params, dt_fixed=0.02)
    return ps


def _lattice_crowded_shell():
    # a cubic lattice with h just below 3 dx: the 30 lattice points at 3 dx fall
    # in every interior particle's shell, more than its 24 slots, so those
    # particles cannot refine and the walk runs
    ps = wl.lattice_block(seed=6, nx=12, ny=12, nz=12, jitter=0.0, h_factor=3.0 * (1.0 - 1e-4))
    ps.v = np.random.default_rng(6).normal(0.0, 0.01, ps.v.shape)
    ps.params = replace(ps.params, dt_fixed=0.01)
    return ps


def _pair_reuse():
    ps = flawed(wl.ceres_pair(seed=4, n_each=2500))
    ps.params = replace(ps.params, dt_fixed=2.0, tree_reuse=2)
    return ps


def _impact_reuse():
    # the measured configuration's physics on a tree reused for 3 steps: the
    # steps after a build refine both evaluations from the build step's walk
    ps = flawed(wl.measurement_1m(seed=35, n_side=18))
    ps.params = replace(ps.params, tree_reuse=3)
    return ps


def _impact_reuse_long():
    # reused for 6 steps with a fixed step 8x the limiter's: the bound fails
    # within the window, and those evaluations walk the widened boxes
    ps = flawed(wl.measurement_1m(seed=37, n_side=14))
    hp = ps.h.min()
    ps.params = replace(ps.params, tree_reuse=6, dt_fixed=0.8 * hp / 64 / (4 * np.sqrt(3)) / 7000.0)
    return ps


CASES = {"impact": _impact, "impact_fast": _impact_fast, "batch": _batch, "rings": _rings,
         "pair_reuse": _pair_reuse, "lattice_crowded_shell": _lattice_crowded_shell,
         "impact_reuse": _impact_reuse, "impact_reuse_long": _impact_reuse_long}


def _run(S, ps, prm, walk_every_eval, nsteps, rk3=False):
    ctx = S.Context(ps.dim, ps.n, max_instances=max(ps.ninst, 1), max_neighbours=160, leaf_size=prm.leaf_size)
    ctx.set_tuning(walk_every_eval=walk_every_eval)
    ds = S.DeviceState(ps)
    ctx.profile(True)
    if rk3:
        dt, t, err, acc = S.step_rk3(ctx, ds, ps.materials, prm, 1e-4, nsteps)
        extra = [dt.cpu().numpy(), t.cpu().numpy(), err.cpu().numpy(), acc.cpu().numpy()]
    else:
        extra = [S.step(ctx, ds, ps.materials, prm, nsteps).cpu().numpy()]
    phases = ctx.profile_read()
    ctx.profile(False)
    return ds.to_numpy(), extra, phases


def _identical(a, b):
    for k in ("x", "v", "rho", "u", "S", "dmg", "h", "id"):
        if a.get(k) is None:
            continue
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", list(CASES))
def test_refined_steps_equal_walked_steps(S, case, prec):
    ps = CASES[case]()
    prm = replace(ps.params, precision=prec)
    R = prm.tree_reuse
    nsteps = 4 if R > 0 else 3
    a, ea, pa = _run(S, ps, prm, 0, nsteps)
    b, eb, pb = _run(S, ps, prm, 1, nsteps)
    _identical(a, b)
    for x, y in zip(ea, eb):
        np.testing.assert_array_equal(x, y)
    # with refinement: a walk at every tree build (each step, or every R-th
    # with a reused tree) and a refine at every other evaluation; without:
    # two walks per step
    builds = nsteps if R == 0 else -(-nsteps // R)
    assert pa["partners"][1] == builds and pa["refine"][1] == 2 * nsteps - builds
    assert pb["refine"][1] == 0 and pb["partners"][1] == 2 * nsteps


def test_refine_bound_holds_and_fails_where_intended(S):
    # the predictor half-step moves every particle by at most dt/2 max|v| per
    # axis (no XSPH): the refined lists are usable where 4 sqrt(3) of that is
    # below h / 64, as in the impact with the limiter's step, and not in the
    # impact with the long fixed step
    for case, usable in (("impact", True), ("impact_fast", False)):
        ps = CASES[case]()
        _, (dt,), _ = _run(S, ps, replace(ps.params, precision="fp64"), 0, 1)
        move = 0.5 * float(dt[0]) * np.abs(ps.v).max()
        ratio = 4 * np.sqrt(3) * move / (ps.h.min() / 64)
        assert (ratio < 0.5) if usable else (ratio > 2), (case, ratio)


def test_crowded_shell_exceeds_its_slots(orc):
    # the lattice case above does overflow the shell (checked by brute force)
    ps = _lattice_crowded_shell()
    off, idx = orc.neighbours(ps.x, ps.h, 3, method="brute")
    offw, idxw = orc.neighbours(ps.x, ps.h * (1.0 + 1.0 / 64.0), 3, method="brute")
    shell = np.diff(offw) - np.diff(off)
    assert shell.max() == 30 and (shell > 24).sum() > 100


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_refined_rk3_equals_walked_rk3(S, prec):
    ps = _impact()
    prm = replace(ps.params, precision=prec)
    a, ea, pa = _run(S, ps, prm, 0, 2, rk3=True)
    b, eb, pb = _run(S, ps, prm, 1, 2, rk3=True)
    _identical(a, b)
    for x, y in zip(ea, eb):
        np.testing.assert_array_equal(x, y)
    assert pa["refine"][1] == 4 and pa["partners"][1] == 2
    assert pb["refine"][1] == 0 and pb["partners"][1] == 6
