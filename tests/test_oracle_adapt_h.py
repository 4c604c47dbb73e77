"""Pins of the oracle's variable smoothing length iteration (Sect. 4.2,
h_new = h (1 + (n_des / n_a)^(1/D)) / 2 with n_a the partners within the
particle's own h): counts against brute force, the closed-form shells of a
cubic lattice, exact single updates and the instance separation."""
import numpy as np
import pytest


def _brute_counts(x, h):
    d = x[:, :, None] - x[:, None, :]
    r2 = (d ** 2).sum(0)
    np.fill_diagonal(r2, np.inf)
    return (r2 < (h ** 2)[:, None]).sum(1)


@pytest.mark.parametrize("dim", [2, 3])
def test_counts_match_brute_force(orc, dim):
    rng = np.random.default_rng(3)
    n = 400
    x = rng.uniform(0, 5, (dim, n))
    h = rng.uniform(0.3, 1.2, n)
    hh, cnt, it = orc.adapt_h(x, h, dim, n_des=20.0, tol=0, max_iter=0)
    assert it == 0
    np.testing.assert_array_equal(hh, h)  # no update with max_iter = 0
    np.testing.assert_array_equal(cnt, _brute_counts(x, h))


def _lattice(m, dim):
    g = np.meshgrid(*([np.arange(m, dtype=float)] * dim), indexing="ij")
    return np.stack([a.ravel() for a in g])


def test_lattice_converges_into_the_shell_interval(orc):
    # unit cubic lattice: shells of 6 at r = 1, 12 at sqrt(2), 8 at sqrt(3), so
    # n_a = 18 exactly for sqrt(2) < h <= sqrt(3)
    m = 12
    x = _lattice(m, 3)
    h = np.full(x.shape[1], 1.2)
    hh, cnt, it = orc.adapt_h(x, h, 3, n_des=18.0, tol=0, max_iter=30)
    inner = np.all((x >= 3) & (x <= m - 4), axis=0)
    assert inner.sum() > 100
    assert (cnt[inner] == 18).all()
    assert (hh[inner] > np.sqrt(2)).all() and (hh[inner] <= np.sqrt(3)).all()
    # boundary particles have no h with exactly 18 partners (counts jump, e.g.
    # 15 -> 19 at a face): the iteration stops at max_iter with them oscillating
    assert it == 30
    assert (hh[~inner] > np.sqrt(2)).all()


def test_exact_single_updates(orc):
    # 3D interior particle with h = 1.8: 6 + 12 + 8 = 26 partners; n_des = 26/8
    # gives (1/8)^(1/3) = 1/2 and h_new = 1.8 * (1 + 1/2) / 2 = 1.35
    x = _lattice(7, 3)
    a = np.flatnonzero(np.all(x == 3, axis=0))[0]
    h = np.full(x.shape[1], 1.8)
    hh, cnt, it = orc.adapt_h(x, h, 3, n_des=26.0 / 8.0, tol=0, max_iter=1)
    assert it == 1 and hh[a] == 1.35
    # 2D: 4 + 4 = 8 partners at h = 1.5; n_des = 2 gives (1/4)^(1/2) = 1/2: 1.125
    x2 = _lattice(7, 2)
    b = np.flatnonzero(np.all(x2 == 3, axis=0))[0]
    hh2, cnt2, _ = orc.adapt_h(x2, np.full(x2.shape[1], 1.5), 2, n_des=2.0, tol=0, max_iter=1)
    assert hh2[b] == 1.125
    # an isolated particle doubles its h
    x3 = np.array([[0.0, 10.0], [0.0, 0.0], [0.0, 0.0]])
    hh3, cnt3, _ = orc.adapt_h(x3, np.array([1.0, 1.0]), 3, n_des=5.0, tol=0, max_iter=1)
    np.testing.assert_array_equal(cnt3, [0, 0])
    np.testing.assert_array_equal(hh3, [2.0, 2.0])


def test_instances_do_not_see_each_other(orc):
    rng = np.random.default_rng(8)
    a = rng.uniform(0, 3, (3, 300))
    b = rng.uniform(0, 3, (3, 200))  # same region of space
    h = rng.uniform(0.4, 0.8, 500)
    x = np.concatenate([a, b], 1)
    off = np.array([0, 300, 500])
    hh, cnt, it = orc.adapt_h(x, h, 3, n_des=12.0, tol=1, max_iter=6, inst_off=off)
    ha, ca, ia = orc.adapt_h(a, h[:300], 3, n_des=12.0, tol=1, max_iter=6)
    hb, cb, ib = orc.adapt_h(b, h[300:], 3, n_des=12.0, tol=1, max_iter=6)
    assert it == max(ia, ib)
    # the instance that converged first keeps iterating with the other one: compare counts of
    # the first pass and the final h of the instance that needed as many updates as the whole
    _, c0, _ = orc.adapt_h(x, h, 3, n_des=12.0, tol=1, max_iter=0, inst_off=off)
    _, c0a, _ = orc.adapt_h(a, h[:300], 3, n_des=12.0, tol=1, max_iter=0)
    _, c0b, _ = orc.adapt_h(b, h[300:], 3, n_des=12.0, tol=1, max_iter=0)
    np.testing.assert_array_equal(c0, np.concatenate([c0a, c0b]))
    if ia == it:
        np.testing.assert_array_equal(hh[:300], ha)
    if ib == it:
        np.testing.assert_array_equal(hh[300:], hb)
