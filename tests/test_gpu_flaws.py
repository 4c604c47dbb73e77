"""Weibull flaw distribution (Sect. 3.2) on the GPU against the oracle: the
CSR offsets bit for bit (they follow from the integer draws alone), the
thresholds to one float ulp (V is summed in a different order and the power
is formed as 2^((log2 j - log2 kV)/m); almost all are bit-equal), on groups
of mixed materials
and instances (sizes 0, 1, 2 and thousands, a non-brittle material, k = 0),
several seeds, a permuted particle order, the 1M-particle measured
configuration and the 256 batched impacts; and the damage model fed with
the GPU's flaws activates as many as with the oracle's."""
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


def _set(n_per_inst, mats_of, seed=0, dim=3):
    rng = np.random.default_rng(seed)
    off = np.concatenate([[0], np.cumsum(n_per_inst)]).astype(np.int64)
    n = int(off[-1])
    mat = np.array([mats_of(i, k) for i, ni in enumerate(n_per_inst) for k in range(ni)], np.int32)
    ids = np.concatenate([off[i] + rng.permutation(ni) for i, ni in enumerate(n_per_inst)]).astype(np.int32)
    x = rng.uniform(0, 1, (dim, n))
    m = rng.uniform(0.5, 2.0, n)
    materials = [wl.Material(rho0=2.7, damage=True, weibull_k=1e12, weibull_m=6.0),
                 wl.Material(rho0=1.0, damage=False),
                 wl.Material(rho0=3.3, damage=True, weibull_k=5e20, weibull_m=9.5)]
    return wl.ParticleSet(dim=dim, x=x, v=np.zeros_like(x), rho=np.ones(n), u=np.zeros(n), m=m, h=np.ones(n),
                          mat=mat, id=ids, inst_off=off if len(n_per_inst) > 1 else None, materials=materials,
                          params=wl.Params(dim=dim))


def _compare(S, orc, ps, seed, **kw):
    ooff, oeps = orc.flaws(ps, seed=seed, **kw)
    ctx = S.Context(ps.dim, max(ps.n, 1), max_instances=max(ps.ninst, 1))
    goff, geps = S.flaws(ctx, S.DeviceState(ps), ps.materials, seed=seed, **kw)
    goff, geps = goff.cpu().numpy(), geps.cpu().numpy()
    np.testing.assert_array_equal(goff, ooff)
    assert len(geps) == len(oeps)
    # one float ulp at most, and almost every value bit-equal
    np.testing.assert_allclose(geps, oeps, rtol=2 ** -23, atol=0)
    assert (geps != oeps).sum() <= 1e-4 * len(oeps) + 2
    return goff, geps


@pytest.mark.parametrize("seed", [0, 77, 2 ** 63 + 5])
def test_mixed_groups_match_oracle(S, orc, seed):
    ps = _set([40, 1, 2, 25, 3000, 600], lambda i, k: (0, 1, 2)[(i + k) % 3] if i not in (1, 2) else 0, seed=3)
    _compare(S, orc, ps, seed)


def test_nonbrittle_and_zero_k(S, orc):
    ps = _set([500, 300], lambda i, k: k % 3, seed=4)
    off, eps = _compare(S, orc, ps, 5, weibull_k=[0.0, 1e30, 5e20], weibull_m=[6.0, 3.0, 9.5])
    nb = _set([50], lambda i, k: 1)
    off, eps = _compare(S, orc, nb, 5)
    assert (off == 0).all() and len(eps) == 0


def test_order_independent(S, orc):
    ps = _set([2000, 1500], lambda i, k: (0, 2)[k % 2], seed=6)
    ctx = S.Context(3, ps.n, max_instances=2)
    a = [t.cpu().numpy() for t in S.flaws(ctx, S.DeviceState(ps), ps.materials, seed=3)]
    rng = np.random.default_rng(1)
    perm = np.concatenate([rng.permutation(2000), 2000 + rng.permutation(1500)])
    ps.x, ps.mat, ps.id, ps.m = ps.x[:, perm], ps.mat[perm], ps.id[perm], ps.m[perm]
    b = [t.cpu().numpy() for t in S.flaws(ctx, S.DeviceState(ps), ps.materials, seed=3)]
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_allclose(a[1], b[1], rtol=2 ** -23, atol=0)


def test_invalid_id_is_reported(S):
    ps = _set([100], lambda i, k: 0, seed=2)
    ps.id = ps.id.copy()
    ps.id[7] = 100  # out of range
    ctx = S.Context(3, ps.n)
    with pytest.raises(S.SphError) as e:
        S.flaws(ctx, S.DeviceState(ps), ps.materials, seed=1)
    assert e.value.status == S.SPH_ERR_INVALID


def test_measured_1m_configuration(S, orc):
    ps = wl.measurement_1m(seed=11, n_side=100)
    ps.flaw_seed = None  # the flaws are what is compared here
    off, eps = _compare(S, orc, ps, 12345)
    assert off[-1] > 14 * ps.n


def test_256_batched_impacts(S, orc):
    ps = wl.batched_impacts(seed=5, with_flaws=False)
    _compare(S, orc, ps, 99)


def test_damage_model_with_gpu_flaws(S, orc):
    # the right-hand side's activated-flaw counts with the GPU's flaws equal the
    # oracle's with its own (the thresholds agree to a float ulp)
    ps = wl.measurement_1m(seed=11, n_side=24)
    ooff, oeps = orc.flaws(ps, seed=8)
    ps.flaw_off, ps.flaw_eps = ooff, oeps
    o = orc.rhs(ps, ps.materials, ps.params)
    ctx = S.Context(3, ps.n, max_neighbours=128, leaf_size=ps.params.leaf_size)
    ds = S.DeviceState(ps)
    ds.flaw_off, ds.flaw_eps = S.flaws(ctx, ds, ps.materials, seed=8)
    g = S.rhs(ctx, ds, ps.materials, replace(ps.params, precision="fp64"))
    np.testing.assert_array_equal(g["n_act"].cpu().numpy(), o["n_act"])


def test_empty_and_single_particle(S, orc):
    e = _set([0], lambda i, k: 0)
    ctx = S.Context(3, 4)
    off, eps = S.flaws(ctx, S.DeviceState(e), e.materials, seed=3)
    assert off.cpu().tolist() == [0] and eps.numel() == 0
    one = _set([1], lambda i, k: 2)
    off, eps = _compare(S, orc, one, 3)
    assert off.tolist() == [0, 1]
