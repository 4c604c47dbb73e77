"""Friends-of-friends fragments (Sect. 4) on the GPU against the oracle:
labels and counts bit for bit (the partition is unique and the numbering is
fixed by count and smallest member), masses to the summation bound
(n_members x 2^-52 relative: both are sums of positive values in different
orders); clustered random sets in 2D and 3D with removed particles, lattice
blocks at the linking length, overlapping instances, min_size 1, an
explicit h0, everything removed, empty and one-particle sets, components all
below min_size, a 2D lattice cut by a damaged line, and the 1M-particle
fragmented body."""
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


def _ps(x, h, m, dmg=None, inst_off=None):
    dim, n = x.shape
    return wl.ParticleSet(dim=dim, x=np.ascontiguousarray(x), v=np.zeros_like(x), rho=np.ones(n), u=np.zeros(n),
                          m=np.ascontiguousarray(m, np.float64), h=np.ascontiguousarray(h, np.float64),
                          mat=np.zeros(n, np.int32), id=np.arange(n, dtype=np.int32), dmg=dmg, inst_off=inst_off,
                          materials=[wl.Material()], params=wl.Params(dim=dim))


def _compare(S, orc, ps, h0=None, link=1.01, d_remove=1.0, min_size=3, kmax=128, depth=21):
    hh = ps.h if h0 is None else h0
    ol, oc, om = orc.fof(ps.x, hh, ps.m, ps.dim, b=link, d_remove=d_remove, min_size=min_size, dmg=ps.dmg,
                         inst_off=ps.inst_off)
    import torch
    ctx = S.Context(ps.dim, max(ps.n, 1), max_instances=max(ps.ninst, 1), max_neighbours=kmax)
    ds = S.DeviceState(ps)
    h0t = None if h0 is None else torch.as_tensor(h0, dtype=torch.float64, device="cuda")
    gl, gc, gm = S.fragments(ctx, ds, h0=h0t, link=link, d_remove=d_remove, min_size=min_size, max_depth=depth)
    gl, gc, gm = gl.cpu().numpy(), gc.cpu().numpy(), gm.cpu().numpy()
    np.testing.assert_array_equal(gc, oc)
    np.testing.assert_array_equal(gl, ol)
    if len(oc):
        np.testing.assert_allclose(gm, om, rtol=float(oc.max()) * 2 ** -52)
    return gl, gc, gm


@pytest.mark.parametrize("dim", [2, 3])
def test_clustered_sets_match_oracle(S, orc, dim):
    rng = np.random.default_rng(30 + dim)
    n = 20000
    centers = rng.uniform(0, 40, (dim, 40))
    x = centers[:, rng.integers(0, 40, n)] + rng.normal(0, 1.5, (dim, n))
    h = rng.uniform(0.3, 0.8, n)
    m = rng.uniform(0.5, 1.5, n)
    dmg = np.where(rng.uniform(size=n) < 0.15, 1.0, rng.uniform(0, 0.99, n))
    _, c, _ = _compare(S, orc, _ps(x, h, m, dmg))
    assert len(c) > 20


@pytest.mark.parametrize("gap", [1.0, 1.02])
def test_lattice_blocks(S, orc, gap):
    g = np.meshgrid(*([np.arange(8, dtype=float)] * 3), indexing="ij")
    a = np.stack([v.ravel() for v in g])
    x = np.concatenate([a, a + np.array([[7 + gap], [0], [0]])], 1)
    n = x.shape[1]
    _, c, _ = _compare(S, orc, _ps(x, np.ones(n), np.ones(n)), depth=10)
    assert c.tolist() == ([1024] if gap == 1.0 else [512, 512])


def test_instances_min_size_and_h0(S, orc):
    rng = np.random.default_rng(5)
    a = rng.uniform(0, 10, (3, 3000))
    b = rng.uniform(2, 12, (3, 2000))
    x = np.concatenate([a, b], 1)
    n = x.shape[1]
    h = rng.uniform(0.5, 1.1, n)
    dmg = rng.uniform(0, 1.2, n)
    ps = _ps(x, h, rng.uniform(1, 2, n), np.minimum(dmg, 1.0), inst_off=np.array([0, 3000, 5000], np.int64))
    _compare(S, orc, ps, depth=20)
    _compare(S, orc, ps, min_size=1, depth=20)
    _compare(S, orc, ps, h0=0.8 * h, d_remove=0.7, depth=20)


def test_everything_removed(S, orc):
    x = np.random.default_rng(2).uniform(0, 3, (3, 500))
    gl, gc, _ = _compare(S, orc, _ps(x, np.ones(500), np.ones(500), np.ones(500)))
    assert len(gc) == 0 and (gl == -1).all()


def test_fragmented_body_1m(S, orc):
    ps = wl.fragmented_body(seed=21)
    assert ps.n == 1_000_000
    _, c, _ = _compare(S, orc, ps)
    assert len(c) > 30


def test_empty_single_and_too_small(S, orc):
    ctx = S.Context(3, 8)
    e = _ps(np.zeros((3, 0)), np.zeros(0), np.zeros(0))
    lab, cnt, mass = S.fragments(ctx, S.DeviceState(e))
    assert lab.numel() == 0 and cnt.numel() == 0
    one = _ps(np.zeros((3, 1)), np.ones(1), np.full(1, 2.0))
    _, c, m = _compare(S, orc, one, min_size=1)
    assert c.tolist() == [1] and m.tolist() == [2.0]
    _, c, _ = _compare(S, orc, one)
    assert len(c) == 0
    # clusters of 5 with min_size 6: nothing qualifies
    x = np.concatenate([np.random.default_rng(1).uniform(0, 0.5, (3, 5)) + 10.0 * k for k in range(6)], 1)
    gl, c, _ = _compare(S, orc, _ps(x, np.ones(30), np.ones(30)), min_size=6)
    assert len(c) == 0 and (gl == -1).all()


def test_2d_damaged_lattice(S, orc):
    g = np.meshgrid(np.arange(60, dtype=float), np.arange(40, dtype=float), indexing="ij")
    x = np.stack([a.ravel() for a in g]) + np.random.default_rng(3).uniform(-0.05, 0.05, (2, 2400))
    dmg = np.where(np.abs(x[0] - 1.3 * x[1] - 5.0) < 1.2, 1.0, 0.3)
    _, c, _ = _compare(S, orc, _ps(x, np.full(2400, 1.2), np.ones(2400), dmg), depth=15)
    assert len(c) >= 2
