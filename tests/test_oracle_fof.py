"""Pins of the oracle's friends-of-friends fragment finder (Sect. 4: fully
damaged particles removed, the rest linked when closer than 1.01 times the
original smoothing length, fragments of fewer than three particles dropped):
brute-force links with scipy's connected components, lattice blocks that join
or separate at the linking length, a chain that breaks where one spacing
exceeds it, a damaged layer that splits a bar, the minimum size, instances
that overlap in space, and mass conservation."""
import math

import numpy as np
import pytest


def _canonical(comp, m, min_size):
    """Fragment labels from component ids: count descending, then smallest
    member index; components below min_size get -1."""
    n = len(comp)
    roots = {}
    for a in range(n):
        if comp[a] >= 0:
            roots.setdefault(comp[a], []).append(a)
    frags = sorted((members for members in roots.values() if len(members) >= min_size),
                   key=lambda mm: (-len(mm), mm[0]))
    label = -np.ones(n, np.int32)
    for f, mm in enumerate(frags):
        label[mm] = f
    return label, np.array([len(mm) for mm in frags], np.int32), np.array([math.fsum(m[mm]) for mm in frags])


def _brute(x, h0, m, b, dmg, d_remove, min_size, inst=None):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    n = x.shape[1]
    hb = b * h0
    d = x[:, :, None] - x[:, None, :]
    r2 = d[0] * d[0] + d[1] * d[1]
    if x.shape[0] == 3:
        r2 = r2 + d[2] * d[2]
    hab = 0.5 * (hb[:, None] + hb[None, :])
    link = r2 < hab * hab
    alive = np.ones(n, bool) if dmg is None else dmg < d_remove
    link &= alive[:, None] & alive[None, :]
    if inst is not None:
        link &= inst[:, None] == inst[None, :]
    np.fill_diagonal(link, False)
    _, cc = connected_components(csr_matrix(link), directed=False)
    comp = np.where(alive, cc, -1)
    return _canonical(comp, m, min_size)


@pytest.mark.parametrize("dim", [2, 3])
def test_matches_brute_force_components(orc, dim):
    rng = np.random.default_rng(10 + dim)
    n = 700
    centers = rng.uniform(0, 12, (dim, 9))
    x = centers[:, rng.integers(0, 9, n)] + rng.normal(0, 0.8, (dim, n))
    h0 = rng.uniform(0.3, 0.7, n)
    m = rng.uniform(0.5, 1.5, n)
    dmg = np.where(rng.uniform(size=n) < 0.2, 1.0, rng.uniform(0, 0.99, n))
    lab, cnt, mass = orc.fof(x, h0, m, dim, b=1.01, d_remove=1.0, min_size=3, dmg=dmg)
    rl, rc, rm = _brute(x, h0, m, 1.01, dmg, 1.0, 3)
    assert len(cnt) > 5 and (lab == -1).sum() > 0.2 * n
    np.testing.assert_array_equal(lab, rl)
    np.testing.assert_array_equal(cnt, rc)
    np.testing.assert_allclose(mass, rm, rtol=n * 2 ** -52)


def _cube(k, origin):
    g = np.meshgrid(*([np.arange(k, dtype=float)] * 3), indexing="ij")
    return np.stack([a.ravel() for a in g]) + np.asarray(origin, float)[:, None]


@pytest.mark.parametrize("gap,joined", [(1.0, True), (1.005, True), (1.02, False), (2.5, False)])
def test_lattice_blocks_join_at_the_linking_length(orc, gap, joined):
    # unit lattice, h0 = 1: neighbours at distance 1 < 1.01 link, diagonals do not matter
    a = _cube(4, (0, 0, 0))
    b = _cube(5, (3 + gap, 0, 0))
    x = np.concatenate([a, b], 1)
    n = x.shape[1]
    lab, cnt, mass = orc.fof(x, np.ones(n), np.ones(n), 3)
    if joined:
        assert cnt.tolist() == [n] and (lab == 0).all()
    else:
        assert cnt.tolist() == [125, 64]
        assert (lab[:64] == 1).all() and (lab[64:] == 0).all()
    np.testing.assert_array_equal(mass, cnt.astype(float))


def test_chain_breaks_where_a_spacing_exceeds_the_link(orc):
    # 2D chain with spacings 1 except one of 1.0101 > 1.01: two fragments
    s = np.ones(19)
    s[7] = 1.0101
    xs = np.concatenate([[0.0], np.cumsum(s)])
    x = np.stack([xs, np.zeros(20)])
    lab, cnt, _ = orc.fof(x, np.ones(20), np.ones(20), 2)
    assert cnt.tolist() == [12, 8]
    assert (lab[:8] == 1).all() and (lab[8:] == 0).all()
    s[7] = 1.0099
    xs = np.concatenate([[0.0], np.cumsum(s)])
    lab, cnt, _ = orc.fof(np.stack([xs, np.zeros(20)]), np.ones(20), np.ones(20), 2)
    assert cnt.tolist() == [20]


def test_damaged_layer_splits_a_bar(orc):
    x = _cube(6, (0, 0, 0))
    n = x.shape[1]
    dmg = np.where(x[0] == 2, 1.0, 0.5)  # the layer x = 2 is fully damaged
    lab, cnt, _ = orc.fof(x, np.ones(n), np.ones(n), 3, dmg=dmg)
    assert cnt.tolist() == [108, 72]
    assert (lab[x[0] == 2] == -1).all()
    assert (lab[x[0] > 2] == 0).all() and (lab[x[0] < 2] == 1).all()
    # nothing survives when everything is damaged
    lab, cnt, mass = orc.fof(x, np.ones(n), np.ones(n), 3, dmg=np.ones(n))
    assert len(cnt) == 0 and (lab == -1).all()


def test_minimum_size(orc):
    # isolated pairs and triples far apart: pairs are dropped with min_size 3
    pts = []
    for k in range(4):
        c = 10.0 * k
        size = 2 if k % 2 == 0 else 3
        pts += [[c + 0.5 * i, 0.0, 0.0] for i in range(size)]
    x = np.array(pts).T
    n = x.shape[1]
    lab, cnt, _ = orc.fof(x, np.ones(n), np.ones(n), 3)
    assert cnt.tolist() == [3, 3]
    assert (lab[:2] == -1).all() and (lab[2:5] == 0).all() and (lab[5:7] == -1).all() and (lab[7:] == 1).all()
    lab, cnt, _ = orc.fof(x, np.ones(n), np.ones(n), 3, min_size=1)
    assert cnt.tolist() == [3, 3, 2, 2]


def test_instances_do_not_link(orc):
    a = _cube(4, (0, 0, 0))
    x = np.concatenate([a, a + 0.3], 1)
    n = x.shape[1]
    off = np.array([0, 64, 128])
    lab, cnt, _ = orc.fof(x, np.ones(n), np.ones(n), 3, inst_off=off)
    assert cnt.tolist() == [64, 64]
    assert (lab[:64] == 0).all() and (lab[64:] == 1).all()
    inst = np.repeat([0, 1], 64)
    rl, rc, _ = _brute(x, np.ones(n), np.ones(n), 1.01, None, 1.0, 3, inst=inst)
    np.testing.assert_array_equal(lab, rl)


def test_mass_is_conserved(orc):
    rng = np.random.default_rng(4)
    x = rng.uniform(0, 6, (3, 900))
    m = rng.uniform(1, 3, 900)
    h0 = np.full(900, 0.9)
    lab, cnt, mass = orc.fof(x, h0, m, 3, min_size=1)
    assert (lab >= 0).all()
    assert abs(mass.sum() - math.fsum(m)) <= 900 * 2 ** -52 * m.sum()
    assert cnt.sum() == 900
