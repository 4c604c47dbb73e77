"""Pins of the oracle's Barnes-Hut evaluation with reused pseudo-particles
(the gravity/hydro decoupling of Sect. 6.3): the tree, node masses and centres
of mass come from the build positions, containment from the particle's
current cell, leaves are summed at current positions.  Pinned by: theta = 0
(no pseudo-particle is used) equals the direct sum at the current positions
whatever the build; build = current positions equals the plain sum; moving
particles inside an accepted far node leaves a distant particle's
acceleration unchanged (the pseudo-particle is frozen) while the fresh sum
changes; an independent numpy rendering of the definition on small sets with
particles moved across cells and out of the root cube; and the step with
reuse equals the step without it when nothing moves."""
from dataclasses import replace

import numpy as np
import pytest

from paper_1604_03290_gb300 import workloads as wl

G, EPS = 1.0, 0.3


def _direct(orc, x, m, h, dim):
    out = orc.gravity_direct(x, m, h, dim, G, EPS)
    return out


def test_theta_zero_is_the_direct_sum_at_current_positions(orc):
    rng = np.random.default_rng(1)
    n = 300
    xb = rng.uniform(0, 1, (3, n))
    x = xb + rng.normal(0, 0.05, (3, n))
    m = rng.uniform(0.5, 1.5, n)
    h = rng.uniform(0.05, 0.1, n)
    a = orc.gravity_bh_reuse(xb, x, m, h, 3, G, 0.0, EPS, 8)
    d = _direct(orc, x, m, h, 3)
    scale = np.abs(d).max()
    np.testing.assert_allclose(a, d, rtol=0, atol=1e-12 * scale)


def test_same_positions_is_the_plain_sum(orc):
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, (2, 400))
    m = np.ones(400)
    h = np.full(400, 0.05)
    np.testing.assert_array_equal(orc.gravity_bh_reuse(x, x, m, h, 2, G, 0.6, EPS, 4),
                                  orc.gravity_bh(x, m, h, 2, G, 0.6, EPS, 4))


def test_far_pseudo_particle_is_frozen(orc):
    # a cluster in [0,1]^3 and one particle at (60,60,60): the level-1 node
    # holding the cluster (edge 30, distance ~103) is accepted at theta 0.5
    rng = np.random.default_rng(3)
    cl = rng.uniform(0, 1, (3, 200))
    xb = np.concatenate([cl, [[60.0], [60.0], [60.0]]], 1)
    n = xb.shape[1]
    m = rng.uniform(0.5, 1.5, n)
    h = np.full(n, 0.1)
    x = xb.copy()
    x[:, :200] += rng.uniform(-0.2, 0.2, (3, 200))  # the cluster moves, its centre of mass too
    reuse = orc.gravity_bh_reuse(xb, x, m, h, 3, G, 0.5, EPS, 8)
    built = orc.gravity_bh(xb, m, h, 3, G, 0.5, EPS, 8)
    fresh = orc.gravity_bh(x, m, h, 3, G, 0.5, EPS, 8)
    np.testing.assert_array_equal(reuse[:, -1], built[:, -1])
    assert np.abs(fresh[:, -1] - built[:, -1]).max() > 1e-6 * np.abs(built[:, -1]).max()
    # and it is the monopole of the cluster as built
    M = m[:200].sum()
    com = (m[:200] * xb[:, :200]).sum(1) / M
    d = x[:, -1] - com
    q = (d ** 2).sum() + (EPS * h[-1]) ** 2
    np.testing.assert_allclose(reuse[:, -1], -G * M * d / q ** 1.5, rtol=1e-12)


def _np_reuse(xb, x, m, h, dim, theta, L, B):
    """The definition, written out: octree of xb (root cube at the per-axis
    minimum, edge = largest extent x (1 + 2^-20); a cell with more than L
    particles above depth B splits into its non-empty octants), node mass and
    centre of mass from xb; each particle's cell from its current position
    (clamped); node used iff its cube does not contain that cell and
    s < theta r; leaves summed at the current positions."""
    n = xb.shape[1]
    lo = xb.min(1)
    s0 = (xb.max(1) - lo).max() * (1 + 2.0 ** -20)
    kb = np.clip(np.floor((xb - lo[:, None]) / s0 * 2.0 ** B), 0, 2 ** B - 1).astype(np.int64)
    kc = np.clip(np.floor((x - lo[:, None]) / s0 * 2.0 ** B), 0, 2 ** B - 1).astype(np.int64)

    def node(level, cell, members):
        mm = m[members]
        return {"level": level, "cell": cell, "members": members, "mass": mm.sum(),
                "com": (mm * xb[:, members]).sum(1) / mm.sum(),
                "leaf": len(members) <= L or level == B, "children": []}

    def split(nd):
        if nd["leaf"]:
            return
        lev = nd["level"] + 1
        sub = {}
        for p in nd["members"]:
            sub.setdefault(tuple(kb[:, p] >> (B - lev)), []).append(p)
        for c in sorted(sub):
            ch = node(lev, np.array(c), np.array(sub[c]))
            split(ch)
            nd["children"].append(ch)

    root = node(0, np.zeros(dim, np.int64), np.arange(n))
    split(root)
    out = np.zeros((dim, n))
    for a in range(n):
        e2 = (EPS * h[a]) ** 2

        def term(xp, mp):
            d = x[:, a] - xp
            q = (d * d).sum() + e2
            return -G * mp * d / q ** 1.5

        def walk(nd):
            inside = np.all((kc[:, a] >> (B - nd["level"])) == nd["cell"])
            if not inside:
                r = np.sqrt(((x[:, a] - nd["com"]) ** 2).sum())
                if s0 / 2.0 ** nd["level"] < theta * r:
                    return term(nd["com"], nd["mass"])
            if nd["leaf"]:
                acc = np.zeros(dim)
                for b in nd["members"]:
                    if b != a:
                        acc += term(x[:, b], m[b])
                return acc
            return sum((walk(c) for c in nd["children"]), np.zeros(dim))

        out[:, a] = walk(root)
    return out


@pytest.mark.parametrize("dim,seed", [(3, 4), (2, 5), (3, 6)])
def test_matches_numpy_rendering(orc, dim, seed):
    rng = np.random.default_rng(seed)
    n = 90
    xb = rng.uniform(0, 1, (dim, n))
    x = xb + rng.normal(0, 0.02, (dim, n))
    x[:, :6] = rng.uniform(0, 1, (dim, 6))  # jump into other cells
    x[:, 6] = xb.max(1) + 0.3  # out of the root cube (clamped cell)
    m = rng.uniform(0.5, 1.5, n)
    h = rng.uniform(0.02, 0.05, n)
    B = 8
    o = orc.gravity_bh_reuse(xb, x, m, h, dim, G, 0.7, EPS, 4, max_depth=B)
    r = _np_reuse(xb, x, m, h, dim, 0.7, 4, B)
    np.testing.assert_allclose(o, r, rtol=0, atol=1e-12 * np.abs(r).max())


def test_step_with_reuse_equals_plain_step_when_nothing_moves(orc):
    # a self-gravitating blob at rest with dt_fixed tiny: the tree of the step
    # start is the tree of every evaluation up to rounding of positions, so one
    # step with tree_reuse 3 equals the plain step to rounding
    ps = wl.lattice_block(seed=3, nx=6, ny=6, nz=6, jitter=0.1)
    ps.params = replace(ps.params, gravity=True, G=1e-3, theta=0.6, dt_fixed=1e-9)
    a, _ = orc.step(ps, ps.materials, ps.params, 2)
    b, _ = orc.step(ps, ps.materials, replace(ps.params, tree_reuse=3), 2)
    for f in ("x", "v", "rho", "u"):
        np.testing.assert_allclose(b[f], a[f], rtol=1e-12, atol=1e-300)
