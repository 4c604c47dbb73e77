"""Pins of the oracle's right-hand side (Sect. 3.1) and predictor-corrector
step (Sect. 3.4.1): linear consistency, co-rotation of stress, conservation
of the symmetric pair forms, signs, limiters, damage and the ring bounce."""
import math
from dataclasses import replace

import numpy as np
import pytest

from paper_1604_03290_gb300 import workloads as wl


def _random_state(seed=0, dim=3, n_side=9, jitter=0.25, strength=True, damage=False):
    ps = wl.lattice_block(seed=seed, nx=n_side, ny=n_side, nz=n_side, dim=dim, jitter=jitter)
    rng = np.random.default_rng(seed + 100)
    n = ps.n
    ps.v = rng.normal(0, 0.05, (dim, n))
    ps.rho = 1.0 + rng.normal(0, 0.02, n)
    ps.u = rng.uniform(0.0, 0.1, n)
    ps.m = ps.m * rng.uniform(0.8, 1.2, n)
    ns = 6 if dim == 3 else 3
    ps.S = rng.normal(0, 0.01, (ns, n)) if strength else None
    if damage:
        import oracle
        ps.dmg = rng.uniform(0, 0.5, n)
        ps.materials = [replace(ps.materials[0], damage=True)]
        ps.flaw_off, ps.flaw_eps = oracle.flaws(ps, weibull_k=[1e8], weibull_m=[6.0], seed=seed + 7)
    return ps


def _spin(dim, omega):
    if dim == 2:
        return np.array([[0.0, -omega], [omega, 0.0]])
    w = np.asarray(omega)
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])


@pytest.mark.parametrize("dim", [2, 3])
def test_corrected_velocity_gradient_is_exact_for_linear_fields(orc, dim):
    ps = _random_state(1, dim, n_side=9 if dim == 3 else 16)
    rng = np.random.default_rng(3)
    G0 = rng.normal(size=(dim, dim))
    ps.v = G0 @ ps.x + rng.normal(size=(dim, 1))
    out = orc.rhs(ps, ps.materials, ps.params)
    gv = out["gradv"].reshape(dim, dim, ps.n)
    assert np.abs(gv - G0[:, :, None]).max() < 1e-11 * np.abs(G0).max()
    # without the correction the boundary particles are badly off
    raw = orc.rhs(ps, ps.materials, replace(ps.params, consistency=False))["gradv"].reshape(dim, dim, ps.n)
    assert np.abs(raw - G0[:, :, None]).max() > 0.1 * np.abs(G0).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_rigid_rotation_co_rotates_the_stress(orc, dim):
    ps = _random_state(2, dim, n_side=8 if dim == 3 else 14)
    n = ps.n
    omega = 0.3 if dim == 2 else np.array([0.1, -0.2, 0.25])
    W = _spin(dim, omega)
    ps.v = W @ ps.x
    rng = np.random.default_rng(4)
    S0 = rng.normal(size=(dim, dim))
    S0 = S0 + S0.T
    S0 -= np.trace(S0) / dim * np.eye(dim)
    comps = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)] if dim == 3 else [(0, 0), (1, 1), (0, 1)]
    ps.S = np.array([np.full(n, S0[i, j]) for i, j in comps]) * 1e-3
    out = orc.rhs(ps, ps.materials, ps.params)
    expect = (W @ S0 - S0 @ W) * 1e-3  # Jaumann: dS/dt = R S - S R, R = spin
    got = out["dS"]
    for k, (i, j) in enumerate(comps):
        assert np.abs(got[k] - expect[i, j]).max() < 1e-12, (i, j)


@pytest.mark.parametrize("dim", [2, 3])
def test_hooke_and_jaumann_for_a_linear_flow(orc, dim):
    # Sect. 2.4: for v = G x + c the corrected gradient is exact, so
    # dS/dt = 2 mu (eps - tr(eps)/D I) + R S - S R with eps = (G + G^T)/2 and
    # R = (G - G^T)/2, for a uniform S (no yield limit, no damage)
    ps = _random_state(21, dim, n_side=9 if dim == 3 else 16)
    n = ps.n
    rng = np.random.default_rng(22)
    G = rng.normal(size=(dim, dim)) * 1e-2
    ps.v = G @ ps.x + rng.normal(size=(dim, 1))
    S0 = rng.normal(size=(dim, dim)) * 1e-3
    S0 = S0 + S0.T
    S0 -= np.trace(S0) / dim * np.eye(dim)
    comps = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)] if dim == 3 else [(0, 0), (1, 1), (0, 1)]
    ps.S = np.array([np.full(n, S0[i, j]) for i, j in comps])
    mu = ps.materials[0].mu
    eps = 0.5 * (G + G.T)
    R = 0.5 * (G - G.T)
    expect = 2 * mu * (eps - np.trace(eps) / dim * np.eye(dim)) + R @ S0 - S0 @ R
    out = orc.rhs(ps, ps.materials, ps.params)
    scale = np.abs(expect).max()
    for k, (i, j) in enumerate(comps):
        assert np.abs(out["dS"][k] - expect[i, j]).max() < 1e-10 * scale, (i, j)


@pytest.mark.parametrize("dim", [2, 3])
def test_deviatoric_rate_is_trace_free(orc, dim):
    ps = _random_state(3, dim, n_side=8 if dim == 3 else 14)
    out = orc.rhs(ps, ps.materials, ps.params)
    tr = out["dS"][:dim].sum(0)
    assert np.abs(tr).max() < 1e-13 * np.abs(out["dS"]).max()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("eps_s", [0.0, 0.2])
def test_total_momentum_conserved(orc, dim, eps_s):
    ps = _random_state(4, dim, n_side=8 if dim == 3 else 14, damage=True)
    ps.rho = 1.0 + np.random.default_rng(5).normal(0, 0.05, ps.n)  # tension and compression
    prm = replace(ps.params, eps_s=eps_s, xsph=0.5)
    out = orc.rhs(ps, ps.materials, prm)
    P = (ps.m * out["dv"]).sum(1)
    assert np.abs(P).max() <= 1e-14 * (ps.m * out["mag_dv"]).sum()
    # XSPH moves the centre of mass with the mean velocity
    assert np.abs((ps.m * (out["dxdt"] - ps.v)).sum(1)).max() <= 1e-15 * (ps.m * np.abs(ps.v)).sum()


@pytest.mark.parametrize("dim", [2, 3])
def test_total_energy_conserved_without_artificial_stress(orc, dim):
    ps = _random_state(5, dim, n_side=8 if dim == 3 else 14, damage=True)
    ps.rho = 1.0 + np.random.default_rng(6).normal(0, 0.05, ps.n)
    out = orc.rhs(ps, ps.materials, ps.params)
    dE = (ps.m * (out["du"] + (ps.v * out["dv"]).sum(0))).sum()
    scale = (ps.m * (out["mag_du"] + np.abs(ps.v).max() * out["mag_dv"])).sum()
    assert abs(dE) <= 1e-14 * scale


def test_angular_momentum_conserved_for_isotropic_forces(orc):
    ps = _random_state(6, 3, n_side=8, strength=False)
    ps.rho = 1.0 + np.random.default_rng(7).normal(0, 0.05, ps.n)
    out = orc.rhs(ps, ps.materials, ps.params)
    Lz = (ps.m * np.cross(ps.x.T, out["dv"].T).T).sum(1)
    scale = (ps.m * np.abs(ps.x).max() * out["mag_dv"]).sum()
    assert np.abs(Lz).max() <= 1e-14 * scale


def test_pressure_repels_and_viscosity_only_for_approach(orc):
    mat = wl.Material(eos="linear", rho0=1.0, cs=1.0)
    base = dict(dim=3, rho=np.array([1.1, 1.1]), u=np.zeros(2), m=np.ones(2), h=np.full(2, 1.0),
                mat=np.zeros(2, np.int32), id=np.arange(2, dtype=np.int32), materials=[mat],
                params=wl.Params(dim=3, alpha=1.0, beta=2.0, consistency=False))
    x = np.array([[0.0, 0.4], [0.0, 0.0], [0.0, 0.0]])
    ps = wl.ParticleSet(x=x, v=np.zeros((3, 2)), **base)
    out = orc.rhs(ps, [mat], ps.params)
    assert out["dv"][0, 0] < 0 < out["dv"][0, 1]  # pushed apart
    # zero pressure: receding pair feels nothing, approaching pair is decelerated
    base["rho"] = np.ones(2)
    rec = wl.ParticleSet(x=x, v=np.array([[-0.1, 0.1], [0, 0], [0, 0]]), **base)
    app = wl.ParticleSet(x=x, v=np.array([[0.1, -0.1], [0, 0], [0, 0]]), **base)
    assert np.abs(orc.rhs(rec, [mat], rec.params)["dv"]).max() == 0.0
    da = orc.rhs(app, [mat], app.params)["dv"]
    assert da[0, 0] < 0 < da[0, 1]
    # and the viscous work heats both (du > 0)
    assert np.all(orc.rhs(app, [mat], app.params)["du"] > 0)


def test_compression_raises_density(orc):
    ps = _random_state(8, 3, n_side=10, strength=False, jitter=0.0)
    c = 0.01
    ps.v = -c * (ps.x - ps.x.mean(1, keepdims=True))
    ps.rho = np.ones(ps.n)
    ps.m = np.ones(ps.n)
    out = orc.rhs(ps, ps.materials, ps.params)
    centre = np.linalg.norm(ps.x - ps.x.mean(1, keepdims=True), axis=0) < 1.5
    # drho/dt = -rho div v = 3 c in the interior of a uniform lattice
    assert np.all(out["drho"][centre] > 0)
    np.testing.assert_allclose(out["drho"][centre], 3 * c, rtol=0.05)


def test_density_sum_on_uniform_lattice(orc):
    ps = _random_state(9, 3, n_side=12, strength=False, jitter=0.0)
    ps.m = np.ones(ps.n)
    ps.rho = np.full(ps.n, 7.0)
    out = orc.rhs(ps, ps.materials, replace(ps.params, density_sum=True))
    centre = np.linalg.norm(ps.x - ps.x.mean(1, keepdims=True), axis=0) < 2.0
    np.testing.assert_allclose(out["rho"][centre], 1.0, rtol=0.02)
    assert np.all(out["drho"] == 0.0)


def test_yield_limiter_written_back_by_the_step(orc):
    ps = _random_state(10, 3, n_side=6)
    mat = replace(ps.materials[0], Y0=0.18)
    ps.materials = [mat]
    ps.S = np.random.default_rng(11).normal(0, 0.05, (6, ps.n))
    full = lambda S: np.array([[S[0], S[3], S[4]], [S[3], S[1], S[5]], [S[4], S[5], S[2]]])
    J2 = np.array([0.5 * (full(ps.S[:, a]) ** 2).sum() for a in range(ps.n)])
    prm = replace(ps.params, dt_fixed=1e-30)
    st, _ = orc.step(ps, [mat], prm, 1)
    J2n = np.array([0.5 * (full(st["S"][:, a]) ** 2).sum() for a in range(ps.n)])
    over = 3 * J2 > mat.Y0 ** 2
    assert over.any() and (~over).any()
    np.testing.assert_allclose(3 * J2n[over], mat.Y0 ** 4 / (3 * J2[over]), rtol=1e-9)
    np.testing.assert_allclose(J2n[~over], J2[~over], rtol=1e-9)


def _isolated_particle(p_target, flaws, mu=1e-8, K=1.0, rho0=1.0, h=0.1, dmg=0.0):
    """One particle with no partner under isotropic tension -p (linear EOS)."""
    mat = wl.Material(eos="linear", rho0=rho0, cs=math.sqrt(K / rho0), K0=K, mu=mu, strength=True, damage=True)
    rho = rho0 + p_target / (K / rho0)
    ps = wl.ParticleSet(dim=3, x=np.zeros((3, 1)), v=np.zeros((3, 1)), rho=np.array([rho]), u=np.zeros(1),
                        m=np.ones(1), h=np.array([h]), mat=np.zeros(1, np.int32), id=np.zeros(1, np.int32),
                        S=np.zeros((6, 1)), dmg=np.array([dmg]), flaw_off=np.array([0, len(flaws)], np.int64),
                        flaw_eps=np.asarray(flaws, np.float32), materials=[mat],
                        params=wl.Params(dim=3, consistency=False))
    return ps, mat


def test_activated_flaw_count(orc):
    K, mu = 2.0, 0.5
    E = 9 * K * mu / (3 * K + mu)
    p = -0.01
    eps = -p / E  # sigma_max = -(1-d) p, eps = sigma_max / ((1-d) E)
    flaws = np.sort(np.array([eps * f for f in (0.2, 0.5, 0.999, 1.001, 1.5, 3.0)], np.float32))
    for dmg in (0.0, 0.6):
        ps, mat = _isolated_particle(p, flaws, mu=mu, K=K, dmg=dmg)
        out = orc.rhs(ps, [mat], ps.params)
        assert out["n_act"][0] == 3
        d = dmg ** 3
        if d < 3 / 6:
            cg = 0.4 * math.sqrt((K + 4 / 3 * (1 - d) * mu) / ps.rho[0])
            assert out["ddmg"][0] == pytest.approx(3 * cg / ps.h[0], rel=1e-14)
    # compression activates nothing
    ps, mat = _isolated_particle(+0.01, flaws, mu=mu, K=K)
    out = orc.rhs(ps, [mat], ps.params)
    assert out["n_act"][0] == 0 and out["ddmg"][0] == 0.0


def test_damage_grows_linearly_until_the_limiter(orc):
    K, mu = 1.0, 1e-8
    eps = 0.01 / (9 * K * mu / (3 * K + mu))
    flaws = np.array([0.1 * eps, 0.2 * eps, 10 * eps, 20 * eps], np.float32)  # two of four activate
    ps, mat = _isolated_particle(-0.01, flaws, mu=mu, K=K, h=0.1)
    cg = 0.4 * math.sqrt(K / ps.rho[0])
    rate = 2 * cg / 0.1
    cap = (2 / 4) ** (1 / 3)
    dt = 0.1 * cap / rate
    st, _ = orc.step(ps, [mat], replace(ps.params, dt_fixed=dt), 5)
    assert st["dmg"][0] == pytest.approx(5 * dt * rate, rel=1e-7)
    st, _ = orc.step(ps, [mat], replace(ps.params, dt_fixed=dt), 40)
    assert st["dmg"][0] == pytest.approx(cap, rel=1e-12)
    # a fully damaged particle carries no tension and activates nothing
    ps, mat = _isolated_particle(-0.01, flaws, mu=mu, K=K, dmg=1.0)
    out = orc.rhs(ps, [mat], ps.params)
    assert out["n_act"][0] == 0


def test_instances_do_not_interact(orc):
    a = _random_state(12, 3, n_side=6)
    both = wl.ParticleSet(dim=3, x=np.concatenate([a.x, a.x], 1), v=np.concatenate([a.v, -a.v], 1),
                          rho=np.concatenate([a.rho, a.rho]), u=np.concatenate([a.u, a.u]),
                          m=np.concatenate([a.m, a.m]), h=np.concatenate([a.h, a.h]),
                          mat=np.zeros(2 * a.n, np.int32), id=np.arange(2 * a.n, dtype=np.int32),
                          S=np.concatenate([a.S, a.S], 1), inst_off=np.array([0, a.n, 2 * a.n]),
                          materials=a.materials, params=a.params)
    o2 = orc.rhs(both, both.materials, both.params)
    o1 = orc.rhs(a, a.materials, a.params)
    np.testing.assert_array_equal(o2["dv"][:, :a.n], o1["dv"])
    np.testing.assert_array_equal(o2["dS"][:, :a.n], o1["dS"])
    assert np.all(o2["nnb"][:a.n] == o1["nnb"])


def test_step_is_second_order_in_time(orc):
    ps = _random_state(13, 2, n_side=12)
    ps.v = ps.v * 2
    T = 0.2
    prm = replace(ps.params, alpha=0.0, beta=0.0)  # no viscosity switch: a smooth right-hand side
    res = {}
    for k in (8, 16, 32, 256):
        st, _ = orc.step(ps, ps.materials, replace(prm, dt_fixed=T / k), k)
        res[k] = np.concatenate([st["x"], st["v"], st["S"]])
    e = [np.abs(res[k] - res[256]).max() for k in (8, 16, 32)]
    # halving dt cuts the error by ~4 for a second-order scheme
    assert 3.3 < e[0] / e[1] < 4.7 and 3.3 < e[1] / e[2] < 4.7


@pytest.mark.slow
def test_rings_bounce_with_artificial_stress(orc):
    """Sect. 4.1 at half resolution: with artificial stress the rings collide,
    reverse and separate as two connected bodies with bounded energy error;
    without it they do not come apart cleanly (the tensile instability)."""
    res = {}
    for AS in (True, False):
        ps = wl.rings_2d(seed=1, dx=0.2, h=0.5, artificial_stress=AS)
        prm = replace(ps.params, dt_fixed=0.3 * 0.5)
        left = ps.x[0] < 0
        E0 = (ps.m * (ps.u + 0.5 * (ps.v ** 2).sum(0))).sum()
        st, _ = orc.step(ps, ps.materials, prm, 1000)
        vl = (ps.m[left] * st["v"][0][left]).sum() / ps.m[left].sum()
        gap = st["x"][0][~left].min() - st["x"][0][left].max()
        E1 = (ps.m * (st["u"] + 0.5 * (st["v"] ** 2).sum(0))).sum()
        off, _ = orc.neighbours(st["x"], ps.h, 2)
        res[AS] = (vl, gap, abs(E1 - E0) / E0, np.diff(off).min())
    vl, gap, dE, nbmin = res[True]
    assert vl < -0.02          # left ring now moves left: the rings bounced
    assert gap > 0.3           # and separated
    assert dE < 0.05
    assert nbmin >= 3          # no particle broke loose
    assert res[False][1] < 0.0  # without artificial stress they are still entangled


def test_xsph_two_particle_closed_form(orc):
    # Sect. 3.1.5: dx_a/dt = v_a + eps sum_b 2 m_b / (rho_a + rho_b) (v_b - v_a) W_ab;
    # for two particles the sum has one term (the kernel itself is pinned above)
    mat = wl.Material(eos="linear", rho0=1.0, cs=1.0)
    for dim in (2, 3):
        x = np.zeros((dim, 2))
        x[0, 1] = 0.37
        v = np.zeros((dim, 2))
        v[:, 0] = 0.3
        v[-1, 1] = -0.2
        rho, m, h = np.array([1.0, 1.4]), np.array([0.7, 1.9]), np.array([1.0, 0.8])
        eps = 0.5
        ps = wl.ParticleSet(dim=dim, x=x, v=v, rho=rho, u=np.zeros(2), m=m, h=h, mat=np.zeros(2, np.int32),
                            id=np.arange(2, dtype=np.int32), materials=[mat],
                            params=wl.Params(dim=dim, consistency=False, xsph=eps))
        out = orc.rhs(ps, [mat], ps.params)
        w = float(orc.W(0.37, 0.9, dim))
        for a, b in ((0, 1), (1, 0)):
            want = v[:, a] + eps * 2 * m[b] / (rho[a] + rho[b]) * (v[:, b] - v[:, a]) * w
            np.testing.assert_allclose(out["dxdt"][:, a], want, rtol=1e-14, atol=1e-16)


@pytest.mark.parametrize("dim", [2, 3])
def test_xsph_vanishes_for_uniform_flow_and_conserves_momentum(orc, dim):
    ps = _random_state(9, dim, n_side=9 if dim == 3 else 20, strength=False)
    ps.params = replace(ps.params, xsph=0.5)
    ps.v = np.repeat(np.array([0.3, -0.2, 0.1])[:dim, None], ps.n, 1)
    out = orc.rhs(ps, ps.materials, ps.params)
    np.testing.assert_array_equal(out["dxdt"], ps.v)  # every difference v_b - v_a is exactly 0
    ps = _random_state(10, dim, n_side=9 if dim == 3 else 20, strength=False)
    ps.params = replace(ps.params, xsph=0.5)
    out = orc.rhs(ps, ps.materials, ps.params)
    corr = out["dxdt"] - ps.v
    # the pair terms are antisymmetric (h_ab, W_ab and the mean density are symmetric)
    tot = (ps.m * corr).sum(1)
    scale = (ps.m * np.abs(corr)).sum(1).max()
    assert scale > 0 and np.abs(tot).max() <= 1e-13 * scale


def _rot3(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.diag(r))


def test_artificial_stress_two_particle_closed_form(orc):
    # Sect. 3.1.4: each particle's tensile principal stresses sigma_i > 0 give
    # zeta_i = -eps_s sigma_i / rho^2 in the principal frame, and the pair adds
    # m_b (zeta_a + zeta_b) f^n grad_a W to dv_a/dt with f = W(r) / W(dmpd);
    # the energy equation does not see it.  Stresses from numpy's eigh, not
    # the oracle's Jacobi rotations.
    rng = np.random.default_rng(12)
    # two materials at their reference densities (zero pressure, so sigma = S)
    mats = [wl.Material(eos="linear", rho0=1.3, cs=1.0, K0=1.0, mu=0.5, strength=True),
            wl.Material(eos="linear", rho0=0.8, cs=1.0, K0=1.0, mu=0.5, strength=True)]
    rho, m, h = np.array([1.3, 0.8]), np.array([0.8, 1.3]), np.array([1.0, 1.2])
    x = np.array([[0.0, 0.45], [0.0, 0.1], [0.0, -0.05]])
    v = np.array([[-0.01, 0.02], [0.0, 0.01], [0.0, 0.0]])  # receding: no artificial viscosity
    S = []
    for a in range(2):
        R = _rot3(rng)
        S.append(R @ np.diag([0.3, -0.05, -0.25] if a == 0 else [0.2, 0.1, -0.3]) @ R.T)
    comp = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    Svec = np.array([[S[a][i, j] for a in range(2)] for i, j in comp])
    eps_s, n_as, dmpd = 0.3, 4.0, 0.5
    base = dict(dim=3, x=x, v=v, rho=rho, u=np.zeros(2), m=m, h=h, S=Svec, mat=np.array([0, 1], np.int32),
                id=np.arange(2, dtype=np.int32), materials=mats)
    p0 = wl.Params(dim=3, consistency=False, n_as=n_as, dmpd=dmpd)
    off = orc.rhs(wl.ParticleSet(params=p0, **base), mats, p0)
    p1 = replace(p0, eps_s=eps_s)
    on = orc.rhs(wl.ParticleSet(params=p1, **base), mats, p1)
    assert (v[:, 0] - v[:, 1]) @ (x[:, 0] - x[:, 1]) > 0
    zeta = []
    for a in range(2):
        lam, Q = np.linalg.eigh(S[a])
        zeta.append(Q @ np.diag(np.where(lam > 0, -eps_s * lam / rho[a] ** 2, 0.0)) @ Q.T)
    d = x[:, 0] - x[:, 1]
    r = np.linalg.norm(d)
    hab = 0.5 * (h[0] + h[1])
    fn = (float(orc.W(r, hab, 3)) / float(orc.W(dmpd, hab, 3))) ** n_as
    g = float(orc.dWdr(r, hab, 3)) * d / r
    for a, b, sgn in ((0, 1, 1.0), (1, 0, -1.0)):
        want = m[b] * (zeta[a] + zeta[b]) @ (sgn * g) * fn
        np.testing.assert_allclose(on["dv"][:, a] - off["dv"][:, a], want, rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(on["du"], off["du"])
    assert np.abs(on["dv"] - off["dv"]).max() > 1e-6  # the term is not negligible here


def test_artificial_viscosity_two_particle_closed_form(orc):
    # Sect. 3.1.3: for an approaching pair nu = h_ab v_ab.x_ab / (r^2 + eps_v h_ab^2),
    # Pi = (-alpha cbar nu + beta nu^2) / rhobar with the mean sound speed and
    # density; with zero stress dv_a/dt = -m_b Pi grad_a W and
    # du_a/dt = 1/2 m_b Pi v_ab.grad_a W
    mats = [wl.Material(eos="linear", rho0=1.3, cs=0.9), wl.Material(eos="linear", rho0=0.8, cs=1.7)]
    rho, m, h = np.array([1.3, 0.8]), np.array([0.8, 1.3]), np.array([1.0, 1.2])
    x = np.array([[0.0, 0.45], [0.0, 0.1], [0.0, -0.05]])
    v = np.array([[0.2, -0.1], [0.05, 0.0], [0.0, 0.03]])
    alpha, beta, eps_v = 1.1, 2.3, 0.01
    prm = wl.Params(dim=3, consistency=False, alpha=alpha, beta=beta, eps_v=eps_v)
    ps = wl.ParticleSet(dim=3, x=x, v=v, rho=rho, u=np.zeros(2), m=m, h=h, mat=np.array([0, 1], np.int32),
                        id=np.arange(2, dtype=np.int32), materials=mats, params=prm)
    out = orc.rhs(ps, mats, prm)
    d, w = x[:, 0] - x[:, 1], v[:, 0] - v[:, 1]
    assert w @ d < 0  # approaching
    r2 = d @ d
    hab = 0.5 * (h[0] + h[1])
    nu = hab * (w @ d) / (r2 + eps_v * hab ** 2)
    Pi = (-alpha * 0.5 * (0.9 + 1.7) * nu + beta * nu ** 2) / (0.5 * (rho[0] + rho[1]))
    g = float(orc.dWdr(np.sqrt(r2), hab, 3)) * d / np.sqrt(r2)
    for a, b, sgn in ((0, 1, 1.0), (1, 0, -1.0)):
        ga = sgn * g
        wab = sgn * w
        np.testing.assert_allclose(out["dv"][:, a], -m[b] * Pi * ga, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(out["du"][a], 0.5 * m[b] * Pi * (wab @ ga), rtol=1e-12)
