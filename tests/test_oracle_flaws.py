"""Pins of the oracle's Weibull flaw distribution (Sect. 3.2, after Benz and
Asphaug): its Philox4x64-10 generator against numpy's independent
implementation; the whole procedure against a plain sequential rendering of
the paper's steps that draws from numpy's Philox; the Weibull law (the r-th
weakest flaw of a group has threshold (r / (k V))^(1/m), i.e. k V eps^m flaws
below eps); coverage (every brittle particle holds a flaw, the last one to be
covered exactly one: the group's strongest); the coupon-collector mean of the
number of flaws, N H_N; independence of the particle order and of the other
groups; and the degenerate groups."""
import math

import numpy as np
import pytest

from paper_1604_03290_gb300 import workloads as wl

M64 = 2 ** 64 - 1


def test_philox_matches_numpy(orc):
    # numpy increments its 256-bit counter before each block: counter c gives block c + 1
    for key, ctr in (([0, 0], 0), ([123, 7], 5), ([M64, 5], M64), ([2 ** 63 + 11, 2 ** 40], (1 << 192) - 1)):
        bg = np.random.Philox(key=np.array(key, np.uint64), counter=ctr)
        raw = [int(v) for v in bg.random_raw(8)]
        c1 = ctr + 1
        c2 = ctr + 2
        w = [(c1 >> (64 * i)) & M64 for i in range(4)]
        w2 = [(c2 >> (64 * i)) & M64 for i in range(4)]
        assert orc.philox4x64(w, key) + orc.philox4x64(w2, key) == raw


def _set(n_per_inst, mats_of, seed=0, dim=3):
    """Particles of several instances; mats_of(i, k) gives the material of the
    k-th particle of instance i."""
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


def _sequential(ps, seed):
    """The procedure of Sect. 3.2 written out step by step, with numpy's
    Philox as the source of the draws."""
    n = ps.n
    off = ps.inst_off if ps.inst_off is not None else np.array([0, n])
    nmat = len(ps.materials)
    lists = [[] for _ in range(n)]  # by id
    for i in range(len(off) - 1):
        for mt, mat in enumerate(ps.materials):
            if not (mat.damage and mat.weibull_k > 0 and mat.weibull_m > 0):
                continue
            mem = [a for a in range(off[i], off[i + 1]) if ps.mat[a] == mt]
            mem.sort(key=lambda a: ps.id[a])
            N = len(mem)
            if N == 0:
                continue
            V = 0.0
            for a in mem:
                V = V + ps.m[a] / mat.rho0
            kV = mat.weibull_k * V
            bg = np.random.Philox(key=np.array([seed, i * nmat + mt], np.uint64), counter=2 ** 256 - 1)
            covered = set()
            j = 0
            while len(covered) < N:
                j += 1
                w = int(bg.random_raw())
                k = (w * N) >> 64
                covered.add(k)
                lists[ps.id[mem[k]]].append(np.float32((j / kV) ** (1.0 / mat.weibull_m)))
    cnt = np.array([len(lst) for lst in lists], np.int64)
    return np.concatenate([[0], np.cumsum(cnt)]), np.array([e for lst in lists for e in lst], np.float32)


@pytest.mark.parametrize("seed", [0, 77, 2 ** 63 + 5])
def test_matches_sequential_procedure_with_numpy_generator(orc, seed):
    ps = _set([40, 1, 25, 60], lambda i, k: (0, 1, 2)[(i + k) % 3] if i != 1 else 0, seed=3)
    off, eps = orc.flaws(ps, seed=seed)
    roff, reps = _sequential(ps, seed)
    np.testing.assert_array_equal(off, roff)
    np.testing.assert_array_equal(eps, reps)


def _groups(ps, off, eps):
    """Per (instance, material) group: the thresholds of its members."""
    io = ps.inst_off if ps.inst_off is not None else np.array([0, ps.n])
    out = {}
    for i in range(len(io) - 1):
        for a in range(io[i], io[i + 1]):
            d = ps.id[a]
            out.setdefault((i, int(ps.mat[a])), []).append(eps[off[d]:off[d + 1]])
    return out


def test_weibull_law(orc):
    # one group of 3000 particles: the r-th weakest flaw is (r / (k V))^(1/m)
    n = 3000
    ps = _set([n], lambda i, k: 0, seed=5)
    mat = ps.materials[0]
    off, eps = orc.flaws(ps, seed=9)
    V = math.fsum(ps.m / mat.rho0)
    s = np.sort(eps.astype(np.float64))
    r = np.arange(1, len(s) + 1)
    np.testing.assert_allclose(s, (r / (mat.weibull_k * V)) ** (1.0 / mat.weibull_m), rtol=2 ** -23)
    # the cumulative number of flaws per volume below eps is k eps^m
    for e in np.quantile(s, [0.1, 0.5, 0.9]) * (1 + 1e-4):
        assert abs((s < e).sum() - mat.weibull_k * V * e ** mat.weibull_m) <= 1.0


def test_coverage_and_order(orc):
    ps = _set([300, 200], lambda i, k: (0, 1, 2)[k % 3], seed=1)
    off, eps = orc.flaws(ps, seed=4)
    cnt = np.diff(off)
    brittle = np.isin(ps.mat, [0, 2])
    by_id = np.empty(ps.n, bool)
    by_id[ps.id] = brittle
    assert (cnt[by_id] >= 1).all() and (cnt[~by_id] == 0).all()
    for d in range(ps.n):
        seg = eps[off[d]:off[d + 1]]
        assert (np.diff(seg) >= 0).all()
    for key, segs in _groups(ps, off, eps).items():
        if key[1] == 1:
            continue
        # the member covered last received exactly one flaw, the group's strongest
        top = max(seg.max() for seg in segs)
        holders = [seg for seg in segs if seg.max() == top]
        assert len(holders) == 1 and len(holders[0]) == 1


def test_coupon_collector_mean(orc):
    # N members need N H_N draws on average (variance ~ pi^2 N^2 / 6)
    N = 400
    tot = []
    for seed in range(48):
        ps = _set([N], lambda i, k: 0, seed=2)
        off, _ = orc.flaws(ps, seed=seed)
        tot.append(off[-1])
    HN = sum(1.0 / k for k in range(1, N + 1))
    sd = math.pi * N / math.sqrt(6.0) / math.sqrt(len(tot))
    assert abs(np.mean(tot) - N * HN) < 4 * sd, (np.mean(tot), N * HN)


def test_independent_of_particle_order_and_other_groups(orc):
    ps = _set([120, 90], lambda i, k: (0, 2)[k % 2], seed=6)
    off, eps = orc.flaws(ps, seed=11)
    # permute within each instance; flaws follow the ids
    rng = np.random.default_rng(1)
    perm = np.concatenate([rng.permutation(120), 120 + rng.permutation(90)])
    q = _set([120, 90], lambda i, k: (0, 2)[k % 2], seed=6)
    q.mat, q.id, q.m = ps.mat[perm], ps.id[perm], ps.m[perm]
    off2, eps2 = orc.flaws(q, seed=11)
    np.testing.assert_array_equal(off, off2)
    np.testing.assert_array_equal(eps, eps2)
    # the first instance alone gets the same flaws
    a = _set([120], lambda i, k: (0, 2)[k % 2], seed=6)
    a.mat, a.id, a.m = ps.mat[:120], ps.id[:120], ps.m[:120]
    offa, epsa = orc.flaws(a, seed=11)
    np.testing.assert_array_equal(offa, off[:121])
    np.testing.assert_array_equal(epsa, eps[:off[120]])


def test_degenerate_groups(orc):
    # no particles
    e = _set([0], lambda i, k: 0)
    off, eps = orc.flaws(e, seed=1)
    assert off.tolist() == [0] and len(eps) == 0
    # nothing brittle
    nb = _set([10], lambda i, k: 1)
    off, eps = orc.flaws(nb, seed=1)
    assert (off == 0).all() and len(eps) == 0
    # a one-particle group takes one flaw: (1 / (k V))^(1/m)
    one = _set([1], lambda i, k: 0)
    mat = one.materials[0]
    off, eps = orc.flaws(one, seed=1)
    assert off.tolist() == [0, 1]
    assert eps[0] == np.float32((1.0 / (mat.weibull_k * (one.m[0] / mat.rho0))) ** (1.0 / mat.weibull_m))
    # a material with k = 0 is not brittle
    off, eps = orc.flaws(one, weibull_k=[0.0, 0.0, 0.0], seed=1)
    assert off.tolist() == [0, 0]
