"""CUDA-graph capture of the step and the autotuner: both must leave every
result bit-identical to plain calls."""
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


def _state_equal(a, b):
    for k in ("x", "v", "rho", "u", "S", "dmg", "id"):
        if a[k] is None:
            continue
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["impact", "batch"])
def test_graph_replay_equals_direct_steps(S, prec, case):
    if case == "impact":
        ps = flawed(wl.measurement_1m(seed=3, n_side=16))
    else:
        ps = flawed(wl.batched_impacts(seed=5, ninst=4, nmin=300, nmax=1200))
        ps.params = replace(ps.params, max_depth=18)
    prm = replace(ps.params, precision=prec)
    ctx1 = S.Context(3, ps.n, max_instances=max(ps.ninst, 1), max_neighbours=160)
    ctx2 = S.Context(3, ps.n, max_instances=max(ps.ninst, 1), max_neighbours=160)
    d1, d2 = S.DeviceState(ps), S.DeviceState(ps)
    S.step(ctx1, d1, ps.materials, prm, 1)  # the graph helper runs one warm-up step
    S.step(ctx1, d1, ps.materials, prm, 3)
    g = S.StepGraph(ctx2, d2, ps.materials, prm, nsteps=1)
    for _ in range(3):
        dt = g.replay()
    import torch
    torch.cuda.synchronize()
    ctx2.sync_status()
    _state_equal(d1.to_numpy(), d2.to_numpy())
    assert np.all(dt.cpu().numpy() > 0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_replay_with_tree_window_equals_direct_steps(S, prec):
    # one tree per 4 steps inside each replay of a 4-step graph (params.tree_reuse):
    # every replay starts its own window, as a 4-step call does
    ps = flawed(wl.batched_impacts(seed=5, ninst=4, nmin=300, nmax=1200))
    prm = replace(ps.params, max_depth=18, precision=prec, tree_reuse=4)
    ctx1 = S.Context(3, ps.n, max_instances=ps.ninst, max_neighbours=160)
    ctx2 = S.Context(3, ps.n, max_instances=ps.ninst, max_neighbours=160)
    d1, d2 = S.DeviceState(ps), S.DeviceState(ps)
    S.step(ctx1, d1, ps.materials, prm, 1)  # the graph helper's warm-up step
    for _ in range(3):
        S.step(ctx1, d1, ps.materials, prm, 4)
    g = S.StepGraph(ctx2, d2, ps.materials, prm, nsteps=4)
    for _ in range(3):
        g.replay()
    import torch
    torch.cuda.synchronize()
    ctx2.sync_status()
    _state_equal(d1.to_numpy(), d2.to_numpy())


def test_autotuner_keeps_results_identical(S, tmp_path):
    from paper_1604_03290_gb300 import autotune
    ps = flawed(wl.measurement_1m(seed=4, n_side=14))
    prm = replace(ps.params, precision="mixed")
    ctx = S.Context(3, ps.n, max_neighbours=160, leaf_size=32)
    ds = S.DeviceState(ps)
    ref = {k: v.cpu().numpy() for k, v in S.rhs(ctx, ds, ps.materials, prm).items()}
    cands = [dict(leaf_size=L, walk_leaf=w, walk_blocks_per_sm=b, pass_threads=t)
             for L, w, b, t in [(8, 32, 8, 64), (32, 256, 24, 128), (16, 64, 16, 128)]]
    prm2, best, ms = autotune.tune(ctx, ds, ps.materials, prm, cache_path=str(tmp_path / "t.json"), cands=cands)
    assert best["walk_leaf"] in (32, 256, 64) and ms > 0
    for c in cands:
        ctx.set_tuning(walk_leaf=c["walk_leaf"], walk_blocks_per_sm=c["walk_blocks_per_sm"],
                       pass_threads=c["pass_threads"])
        out = {k: v.cpu().numpy() for k, v in
               S.rhs(ctx, ds, ps.materials, replace(prm, leaf_size=c["leaf_size"])).items()}
        for k in ("dv", "du", "drho", "dS", "ddmg", "n_act", "nnb"):
            np.testing.assert_array_equal(out[k], ref[k], err_msg=(k, c))
    # cached
    prm3, best3, _ = autotune.tune(ctx, ds, ps.materials, prm, cache_path=str(tmp_path / "t.json"))
    assert best3 == best


@pytest.mark.parametrize("case", ["impact", "cloud", "ceres"])
def test_plain_forms_equal_fused_forms(S, case):
    """sph_tuning.plain_forms = 1 packs the FP32 views in a separate launch at
    every evaluation and reads the gravity walk's node records unpacked; the
    default writes the views in the update on a kept tree and reads the packed
    node word.  Steps on a reused tree must give the same states bit for bit."""
    if case == "impact":
        ps = flawed(wl.measurement_1m(seed=5, n_side=18))
        prm = replace(ps.params, precision="mixed", tree_reuse=4)
    elif case == "cloud":  # variable h: a tree per step, the packed gravity word
        ps = wl.cloud_collapse(seed=3, n=30_000)
        prm = replace(ps.params, precision="mixed", tree_reuse=3)
    else:  # gravity on a kept tree: both forms at once
        ps = flawed(wl.ceres_pair(seed=4, n_each=15_000))
        prm = replace(ps.params, precision="mixed", tree_reuse=3)
    out = []
    for plain in (0, 1):
        ctx = S.Context(3, ps.n, max_neighbours=160, leaf_size=ps.params.leaf_size)
        ctx.set_tuning(plain_forms=plain)
        assert ctx.get_tuning()["plain_forms"] == plain
        ds = S.DeviceState(ps)
        S.step(ctx, ds, ps.materials, prm, 7)
        out.append(ds.to_numpy())
    _state_equal(out[0], out[1])
