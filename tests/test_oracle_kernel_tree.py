"""Pins of the oracle's kernel (Sect. 3.1.1), partner search (Sect. 3.5.2)
and octree (Sect. 3.5.1) against closed forms, brute force and scipy."""
import math
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.spatial import cKDTree

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_norm():
    out = {}
    for line in open(os.path.join(GOLDEN, "kernel_normalisation.txt")):
        if line.startswith("#") or not line.strip():
            continue
        d, _, v = line.split()
        out[int(d)] = float(v)
    return out


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_kernel_normalisation_constant_matches_paper(orc, dim):
    assert orc.W(0.0, 1.0, dim) == pytest.approx(_golden_norm()[dim], rel=1e-15)


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("h", [1.0, 0.37, 5.0])
def test_kernel_integrates_to_one(orc, dim, h):
    shell = {1: lambda r: 2.0, 2: lambda r: 2.0 * math.pi * r, 3: lambda r: 4.0 * math.pi * r * r}[dim]
    f = lambda r: orc.W(r, h, dim) * shell(r)
    val = integrate.quad(f, 0.0, h / 2, epsabs=1e-14, epsrel=1e-13)[0] + \
        integrate.quad(f, h / 2, h, epsabs=1e-14, epsrel=1e-13)[0]
    assert val == pytest.approx(1.0, abs=1e-11)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_kernel_derivative_is_derivative(orc, dim):
    h = 0.8
    for r in np.linspace(0.01, 0.99, 57) * h:
        eps = 1e-6 * h
        fd = (orc.W(r + eps, h, dim) - orc.W(r - eps, h, dim)) / (2 * eps)
        assert orc.dWdr(r, h, dim) == pytest.approx(fd, rel=1e-7, abs=1e-9)


@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_continuity_and_support(orc, dim):
    h = 1.3
    for f in (orc.W, orc.dWdr):
        a, b = f(0.5 * h * (1 - 1e-12), h, dim), f(0.5 * h * (1 + 1e-12), h, dim)
        assert a == pytest.approx(b, rel=1e-9)
        assert f(h, h, dim) == 0.0
        assert f(1.0001 * h, h, dim) == 0.0
    assert orc.dWdr(0.0, h, dim) == 0.0


def _random_points(rng, n, dim, box=10.0):
    return rng.uniform(0, box, size=(dim, n))


@pytest.mark.parametrize("dim", [2, 3])
def test_brute_partners_match_kdtree(orc, dim):
    rng = np.random.default_rng(7)
    n = 1500
    x = _random_points(rng, n, dim, box=12.0 if dim == 3 else 30.0)
    h = np.full(n, 1.3)
    off, idx = orc.neighbours(x, h, dim, method="brute")
    t = cKDTree(x.T)
    for a in range(n):
        cand = np.array(sorted(t.query_ball_point(x[:, a], 1.3)))
        d = np.sqrt(((x[:, cand] - x[:, [a]]) ** 2).sum(0))
        ref = cand[(d < 1.3) & (cand != a)]
        np.testing.assert_array_equal(idx[off[a]:off[a + 1]], ref)


@pytest.mark.parametrize("dim", [2, 3])
def test_grid_partners_equal_brute_force_variable_h(orc, dim):
    rng = np.random.default_rng(8)
    n = 2500
    x = _random_points(rng, n, dim, box=10.0 if dim == 3 else 25.0)
    h = rng.uniform(0.6, 1.8, n)
    o1, i1 = orc.neighbours(x, h, dim, method="brute")
    o2, i2 = orc.neighbours(x, h, dim, method="grid")
    np.testing.assert_array_equal(o1, o2)
    np.testing.assert_array_equal(i1, i2)
    # symmetric, sorted, no self
    pairs = set()
    for a in range(n):
        lst = i1[o1[a]:o1[a + 1]]
        assert np.all(np.diff(lst) > 0) and a not in lst
        pairs.update((a, int(b)) for b in lst)
    assert all((b, a) in pairs for a, b in pairs)
    for a in rng.integers(0, n, 20):
        np.testing.assert_array_equal(orc.neighbours_one(x, h, dim, int(a)), i1[o1[a]:o1[a + 1]])


def test_partner_uses_mean_smoothing_length_and_strict_bound(orc):
    h = np.array([1.0, 3.0])
    for r, expect in [(1.9, 1), (2.0, 0), (2.1, 0)]:
        x = np.array([[0.0, r], [0.0, 0.0], [0.0, 0.0]])
        off, idx = orc.neighbours(x, h, 3, method="brute")
        assert off[-1] == 2 * expect


def _cells(k, level, B):
    return k >> (B - level)


@pytest.mark.parametrize("dim,L", [(3, 1), (3, 8), (2, 4), (3, 16)])
def test_octree_nodes_match_enumeration(orc, dim, L):
    rng = np.random.default_rng(9)
    n = 3000
    x = rng.normal(size=(dim, n)) ** 3  # clustered: deep chains
    x[:, :5] = x[:, [5]]  # coincident particles reach full depth
    m = rng.uniform(0.5, 2.0, n)
    B = 21
    T = orc.tree_nodes(x, m, dim, L, B)
    k = orc.cell_coords(x, dim, B)[:, :dim]
    # enumerate every cell that must be a node: root, and every non-empty cell
    # whose parent holds more than L particles (and lies above full depth)
    expect = {}
    for lev in range(B + 1):
        c = _cells(k, lev, B)
        keys, inv, cnt = np.unique(c, axis=0, return_inverse=True, return_counts=True)
        if lev == 0:
            parent_ok = np.ones(len(keys), bool)
        else:
            pc = _cells(k, lev - 1, B)
            pk, pinv, pcnt = np.unique(pc, axis=0, return_inverse=True, return_counts=True)
            first = np.zeros(len(keys), np.int64)
            first[inv.ravel()] = np.arange(n)
            parent_ok = pcnt[pinv.ravel()[first]] > L
        for kk, cc, ok in zip(map(tuple, keys), cnt, parent_ok):
            if ok:
                expect[(lev,) + kk] = cc
    got = {(int(l),) + tuple(int(v) for v in c[:dim]): int(cnt)
           for l, c, cnt in zip(T["level"], T["cell"], T["count"])}
    assert got == expect
    # mass and centre of mass of every node straight from its particles
    for i in rng.integers(0, len(T["level"]), 200):
        lev = int(T["level"][i])
        sel = np.all(_cells(k, lev, B) == T["cell"][i, :dim], axis=1)
        assert T["mass"][i] == pytest.approx(m[sel].sum(), rel=1e-13)
        np.testing.assert_allclose(T["com"][i, :dim], (x[:, sel] * m[sel]).sum(1) / m[sel].sum(),
                                   rtol=1e-12, atol=1e-12 * np.abs(x).max())
    # pre-order: a node's subtree follows it contiguously
    lev = T["level"]
    assert lev[0] == 0 and np.all(lev[1:] <= np.maximum.accumulate(lev)[:-1] + 1)


def test_cell_coordinates_cover_root_cube(orc):
    rng = np.random.default_rng(10)
    x = rng.uniform(-3, 5, size=(3, 500))
    k = orc.cell_coords(x, 3, 21)
    assert k.min() >= 0 and k.max() <= (1 << 21) - 1
    # the largest extent axis spans (almost) the full index range
    assert k[:, 0].max() > (1 << 21) - 10 or k[:, 1].max() > (1 << 21) - 10 or k[:, 2].max() > (1 << 21) - 10
