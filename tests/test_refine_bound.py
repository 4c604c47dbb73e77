"""The bound behind refining partner lists within a step (CPU, with the
oracle's brute-force partner search).  Partners are N(a) = {b != a : r_ab <
h_ab}, h_ab = (h_a + h_b)/2 (Sect. 3.5.2).  A walk at positions x records
N(a) and the shell {b : (1 - 1/64) h_ab <= r_ab < (1 + 1/64) h_ab}; if every
particle then moves by at most `move` per axis with 4 sqrt(D) move <= h_a / 64
for every a, each partner at the new positions must be in N(a) or the shell,
and each partner closer than (1 - 1/64) h_ab must still be a partner: the
library then re-tests only the shell's members instead of walking the tree
again.  Checked on clustered sets with variable h in 2D and 3D, with random
moves at the bound, with pairs just outside (inside) the shell pushed together
(apart) as far as the bound allows, and shown to fail when the moves are 8
times larger."""
import numpy as np
import pytest

SKIN = 1.0 / 64.0


def _sets(orc, x, h, dim):
    off, idx = orc.neighbours(x, h, dim, method="brute")
    return [set(idx[off[a]:off[a + 1]].tolist()) for a in range(x.shape[1])]


def _candidates(orc, x, h, dim):
    # partners and shell together: b != a with r_ab < (1 + skin) h_ab, taken a
    # hair wider so that rounding of the scaled h cannot drop a member
    return _sets(orc, x, h * (1.0 + SKIN) * (1.0 + 1e-12), dim)


def _deep(orc, x, h, dim):
    # partners closer than (1 - skin) h_ab, taken a hair narrower
    return _sets(orc, x, h * (1.0 - SKIN) * (1.0 - 1e-12), dim)


def _clustered(rng, dim, n):
    centres = rng.uniform(0, 6, (dim, 12))
    x = centres[:, rng.integers(0, 12, n)] + rng.normal(0, 0.8, (dim, n))
    h = rng.uniform(0.25, 0.6, n)
    return x, h


@pytest.mark.parametrize("dim,seed", [(3, 1), (3, 2), (2, 3)])
def test_partners_after_bounded_moves_are_candidates(orc, dim, seed):
    rng = np.random.default_rng(seed)
    n = 2500
    x, h = _clustered(rng, dim, n)
    cand = _candidates(orc, x, h, dim)
    deep = _deep(orc, x, h, dim)
    move = h.min() * SKIN / (4.0 * np.sqrt(dim))
    for trial in range(3):
        y = x + rng.uniform(-move, move, (dim, n))
        y[:, : n // 4] = x[:, : n // 4] + move * rng.choice([-1.0, 1.0], (dim, n // 4))  # corners of the box
        new = _sets(orc, y, h, dim)
        missing = sum(len(new[a] - cand[a]) for a in range(n))
        assert missing == 0, (trial, missing)
        lost = sum(len(deep[a] - new[a]) for a in range(n))
        assert lost == 0, (trial, lost)
        # and the new partners changed at all (the moves are not vacuous)
        old = _sets(orc, x, h, dim)
        assert sum(len(new[a] ^ old[a]) for a in range(n)) > 0


def test_pairs_just_outside_the_shell_stay_apart(orc):
    # two particles at (1 + skin) h_ab (1 + 1e-9), pushed straight at each other
    # by the largest move the bound allows on every axis: still no partners
    dim = 3
    for ha, hb in ((1.0, 1.0), (1.0, 0.3), (0.3, 1.0)):
        hab = 0.5 * (ha + hb)
        r = (1.0 + SKIN) * hab * (1.0 + 1e-9)
        d = np.array([1.0, 1.0, 1.0]) / np.sqrt(3.0)
        x = np.stack([np.zeros(3), r * d], 1)
        h = np.array([ha, hb])
        move = min(ha, hb) * SKIN / (4.0 * np.sqrt(dim))
        y = x + np.stack([move * np.ones(3), -move * np.ones(3)], 1)
        assert _sets(orc, x, h, dim)[0] == set()
        assert _sets(orc, y, h, dim)[0] == set()
        assert np.linalg.norm(y[:, 1] - y[:, 0]) < r  # they did come closer


def test_pairs_just_inside_the_shell_stay_partners(orc):
    # two particles at (1 - skin) h_ab (1 - 1e-9), pulled straight apart by the
    # largest move the bound allows on every axis: still partners
    dim = 3
    for ha, hb in ((1.0, 1.0), (1.0, 0.3), (0.3, 1.0)):
        hab = 0.5 * (ha + hb)
        r = (1.0 - SKIN) * hab * (1.0 - 1e-9)
        d = np.array([1.0, 1.0, 1.0]) / np.sqrt(3.0)
        x = np.stack([np.zeros(3), r * d], 1)
        h = np.array([ha, hb])
        move = min(ha, hb) * SKIN / (4.0 * np.sqrt(dim))
        y = x + np.stack([-move * np.ones(3), move * np.ones(3)], 1)
        assert _sets(orc, x, h, dim)[0] == {1}
        assert _sets(orc, y, h, dim)[0] == {1}
        assert np.linalg.norm(y[:, 1] - y[:, 0]) > r  # they did move apart


def test_larger_moves_break_the_bound(orc):
    # with moves 8 times the bound some new partner lies outside the old
    # partners and shell: the bound is what makes the refinement exact
    rng = np.random.default_rng(5)
    dim, n = 3, 2500
    x, h = _clustered(rng, dim, n)
    cand = _candidates(orc, x, h, dim)
    move = 8.0 * h.min() * SKIN / (4.0 * np.sqrt(dim))
    y = x + move * rng.choice([-1.0, 1.0], (dim, n))
    new = _sets(orc, y, h, dim)
    assert sum(len(new[a] - cand[a]) for a in range(n)) > 0
    deep = _deep(orc, x, h, dim)
    assert sum(len(deep[a] - new[a]) for a in range(n)) > 0
