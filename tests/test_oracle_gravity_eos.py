"""Pins of the oracle's gravity (Sect. 3.3), equations of state (Sect. 2.5),
the principal-axis solve (Sect. 3.2) and the paper's printed constants."""
import math
import os

import numpy as np
import pytest

from paper_1604_03290_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_two_body_closed_form(orc):
    x = np.array([[0.0, 3.0], [0.0, 4.0], [0.0, 0.0]])
    m = np.array([2.0, 5.0])
    h = np.array([0.2, 0.4])
    G, eg = 1.5, 0.5
    for a in (orc.gravity_direct(x, m, h, 3, G, eg), orc.gravity_bh(x, m, h, 3, G, 0.5, eg, 1)):
        e0, e1 = eg * h[0], eg * h[1]
        # particle 0 pulled towards particle 1 with |a| = G m1 r / (r^2 + e^2)^1.5
        np.testing.assert_allclose(a[:, 0], G * 5.0 * np.array([3.0, 4.0, 0.0]) / (25.0 + e0 ** 2) ** 1.5, rtol=1e-14)
        np.testing.assert_allclose(a[:, 1], -G * 2.0 * np.array([3.0, 4.0, 0.0]) / (25.0 + e1 ** 2) ** 1.5, rtol=1e-14)


@pytest.mark.parametrize("dim,L", [(3, 1), (3, 16), (2, 4)])
def test_tree_at_zero_opening_angle_is_direct_sum(orc, dim, L):
    rng = np.random.default_rng(11)
    n = 1200
    x = rng.normal(size=(dim, n))
    m = rng.uniform(0.5, 1.5, n)
    h = rng.uniform(0.05, 0.2, n)
    d = orc.gravity_direct(x, m, h, dim, 1.0, 0.5)
    b = orc.gravity_bh(x, m, h, dim, 1.0, 0.0, 0.5, L)
    scale = np.abs(d).max()
    assert np.abs(b - d).max() <= 1e-13 * scale


def test_direct_sum_conserves_momentum_with_uniform_softening(orc):
    rng = np.random.default_rng(12)
    n = 800
    x = rng.normal(size=(3, n))
    m = rng.uniform(0.5, 1.5, n)
    h = np.full(n, 0.1)
    a = orc.gravity_direct(x, m, h, 3, 1.0, 0.5)
    assert np.abs((m * a).sum(1)).max() <= 1e-13 * (m * np.abs(a)).sum()


def test_uniform_ball_interior_field(orc):
    """Inside a uniform ball g(r) = -(4/3) pi G rho r."""
    dx = 1.0
    R = 18.0
    ps_x = wl._lattice_ball(R, dx)
    n = ps_x.shape[1]
    rho = 1.0
    m = np.full(n, rho * dx ** 3)
    h = np.full(n, 2.4 * dx)
    r = np.sqrt((ps_x ** 2).sum(0))
    sample = np.where((r > 0.3 * R) & (r < 0.6 * R))[0][::37]
    a = orc.gravity_bh(ps_x, m, h, 3, 1.0, 0.4, 0.5, 8, sample=sample)
    expect = -(4.0 / 3.0) * math.pi * rho * ps_x[:, sample]
    err = np.sqrt(((a - expect) ** 2).sum(0)) / np.sqrt((expect ** 2).sum(0))
    assert err.max() < 0.03


def test_barnes_hut_error_falls_with_opening_angle(orc):
    rng = np.random.default_rng(13)
    n = 4000
    x = rng.normal(size=(3, n))
    m = np.ones(n)
    h = np.full(n, 0.05)
    d = orc.gravity_direct(x, m, h, 3, 1.0, 0.5)
    errs = []
    for th in (0.2, 0.4, 0.8):
        b = orc.gravity_bh(x, m, h, 3, 1.0, th, 0.5, 1)
        errs.append(np.sqrt(((b - d) ** 2).sum(0)).mean() / np.sqrt((d ** 2).sum(0)).mean())
    assert errs[0] < errs[1] < errs[2]
    # error grows about as theta^2 (monopoles, Sect. 3.3): ratio 4 per doubling
    assert 2.0 < errs[2] / errs[1] < 10.0
    assert errs[2] < 0.05


def _golden_materials():
    out = {}
    for line in open(os.path.join(GOLDEN, "materials.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, key, val = line.split()
        out.setdefault(name, {})[key] = float(val)
    return out


def test_material_tables_transcribed(orc):
    g = _golden_materials()
    mats = {"Al6061": wl.aluminium_6061(), "basalt": wl.basalt(), "ice": wl.ice(), "rubber": wl.rubber()}
    for name, vals in g.items():
        for k, v in vals.items():
            assert getattr(mats[name], k) == pytest.approx(v, rel=1e-12), (name, k)


def test_cloud_free_fall_time_and_sound_speed():
    g = {}
    for line in open(os.path.join(GOLDEN, "cloud_collapse.txt")):
        if not line.startswith("#") and line.strip():
            k, v = line.split()
            g[k] = float(v)
    tff = math.sqrt(3 * math.pi / (32 * wl.G_SI * g["rho0"]))
    assert tff == pytest.approx(g["t_ff"], rel=2e-3)  # the paper's G differs in the 4th digit
    mat = wl.molecular_hydrogen_10K()
    assert mat.rho0 == g["rho0"]
    assert mat.cs == pytest.approx(203.1, rel=1e-3)
    # mass of the uniform cloud: 4/3 pi R0^3 rho0 ~ 1 M_sun
    assert 4 / 3 * math.pi * g["R0"] ** 3 * g["rho0"] / wl.M_SUN == pytest.approx(1.0, rel=0.02)


def test_eos_zero_pressure_at_reference_state(orc):
    for mat in (wl.aluminium_6061(), wl.basalt(), wl.ice(), wl.rubber(),
                wl.Material(eos="murnaghan", rho0=2.0, K0=3.0, n_M=4.0)):
        p = orc.eos(mat, mat.rho0, 0.0)[0]
        assert p == 0.0


def test_linear_equals_murnaghan_with_unit_exponent(orc):
    lin = wl.Material(eos="linear", rho0=1.3, cs=2.0)
    mur = wl.Material(eos="murnaghan", rho0=1.3, K0=1.3 * 4.0, n_M=1.0)
    for rho in (0.7, 1.0, 1.3, 2.2):
        a, b = orc.eos(lin, rho, 0.0), orc.eos(mur, rho, 0.0)
        assert a[0] == pytest.approx(b[0], rel=1e-14, abs=1e-14)
        assert a[3] == pytest.approx(b[3], rel=1e-14)


def test_linear_cutoff(orc):
    lin = wl.Material(eos="linear", rho0=1.0, cs=1.0, rho_cut=0.9)
    assert orc.eos(lin, 0.95, 0)[0] == pytest.approx(-0.05)
    assert orc.eos(lin, 0.85, 0)[0] == 0.0


def test_isothermal_is_ideal_gas(orc):
    mat = wl.molecular_hydrogen_10K()
    for rho in (1e-15, 1e-14, 1e-12):
        p, _, _, c = orc.eos(mat, rho, 0.0)
        assert p == pytest.approx(rho * mat.cs ** 2, rel=1e-15)
        assert c == pytest.approx(mat.cs, rel=1e-15)


@pytest.mark.parametrize("mat", [wl.aluminium_6061(), wl.basalt(), wl.ice()], ids=lambda m: m.name)
def test_tillotson_continuity_at_branch_joins(orc, mat):
    rho0 = mat.rho0
    for eta in (0.6, 0.9, 0.99):
        rho = eta * rho0
        for u in (mat.E_iv, mat.E_cv):
            lo, hi = orc.eos(mat, rho, u * (1 - 1e-12))[0], orc.eos(mat, rho, u * (1 + 1e-12))[0]
            assert lo == pytest.approx(hi, rel=1e-8, abs=1e-8 * mat.A_T)
    for u in (0.5 * mat.E_iv, 0.5 * (mat.E_iv + mat.E_cv), 2 * mat.E_cv):
        lo, hi = orc.eos(mat, rho0 * (1 - 1e-13), u)[0], orc.eos(mat, rho0, u)[0]
        assert lo == pytest.approx(hi, rel=1e-8, abs=1e-8 * mat.A_T)


@pytest.mark.parametrize("mat", [wl.aluminium_6061(), wl.basalt()], ids=lambda m: m.name)
def test_tillotson_derivatives_match_finite_differences(orc, mat):
    rho0 = mat.rho0
    pts = [(1.2, 0.3), (1.05, 2.0), (0.8, 0.3), (0.8, 0.5 * (mat.E_iv + mat.E_cv) / mat.E_iv), (0.5, 3 * mat.E_cv / mat.E_iv)]
    for eta, uu in pts:
        rho, u = eta * rho0, uu * mat.E_iv
        p, pr, pu, c = orc.eos(mat, rho, u)
        dr, du = 1e-6 * rho, 1e-6 * u
        fr = (orc.eos(mat, rho + dr, u)[0] - orc.eos(mat, rho - dr, u)[0]) / (2 * dr)
        fu = (orc.eos(mat, rho, u + du)[0] - orc.eos(mat, rho, u - du)[0]) / (2 * du)
        assert pr == pytest.approx(fr, rel=1e-6, abs=1e-9 * mat.A_T / rho0)
        assert pu == pytest.approx(fu, rel=1e-6, abs=1e-9 * rho0)
        c2 = max(mat.A_T / rho0, pr + p / rho ** 2 * pu)
        assert c * c == pytest.approx(c2, rel=1e-12)


def test_tillotson_limits(orc):
    mat = wl.aluminium_6061()
    # cold compression curve: u = 0 gives A chi + B chi^2
    for eta in (1.01, 1.2, 1.5):
        chi = eta - 1
        assert orc.eos(mat, eta * mat.rho0, 0.0)[0] == pytest.approx(mat.A_T * chi + mat.B_T * chi ** 2, rel=1e-13)
    # strongly expanded hot gas tends to the ideal gas p = a rho u
    rho, u = 0.01 * mat.rho0, 50 * mat.E_cv
    assert orc.eos(mat, rho, u)[0] == pytest.approx(mat.a_T * rho * u, rel=1e-6)


@pytest.mark.parametrize("dim", [2, 3])
def test_jacobi_principal_axes(orc, dim):
    rng = np.random.default_rng(14)
    for _ in range(200):
        A = rng.normal(size=(dim, dim)) * 10 ** rng.uniform(-3, 9)
        A = A + A.T
        w, V = orc.sym_eig(A)
        ref = np.linalg.eigvalsh(A)
        scale = np.abs(ref).max()
        assert np.abs(w - ref).max() <= 1e-13 * scale
        assert np.abs(V.T @ V - np.eye(dim)).max() <= 1e-13
        assert np.abs(A @ V - V * w).max() <= 1e-12 * scale
    w, _ = orc.sym_eig(np.diag([3.0, -1.0, 2.0][:dim]))
    np.testing.assert_array_equal(w, np.sort(np.array([3.0, -1.0, 2.0][:dim])))
