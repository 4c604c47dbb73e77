"""Pins of the oracle's Tillotson expanded branch (Sect. 2.5.3, Eq. tillo2).

The continuity and derivative pins elsewhere leave the two exponentials of the
expanded form free: at rho = rho0 both are 1, far out both vanish, and the
branch join holds by the interpolation.  The tests here fix them separately,
at interior points of the expanded region (rho < rho0, u >= E_cv) where
orc_eos returns the expanded pressure p_e unmixed.

With eta = rho/rho0, chi = eta - 1, z = rho0/rho - 1 and omega = 1 + u/(E0 eta^2)
the equation reads

    p_e = a rho u + [ b rho u / omega + A chi exp(-beta z) ] exp(-alpha z^2).

Two consequences of that structure, each checked on its own:

* the u-dependent part: at fixed rho, p_e(u1) - p_e(u2) - a rho (u1 - u2)
  = b rho (u1/omega1 - u2/omega2) exp(-alpha z^2).  The log of the ratio is
  a pure quadratic in z whose coefficient is -alpha (no constant, no linear
  term).  A dropped square, alpha and beta exchanged, or the alpha factor
  misplaced outside the bracket gives a constant or linear term instead.
* the cold part: (p_e - a rho u) exp(+alpha z^2) - b rho u/omega
  = A chi exp(-beta z); log of it over A chi is linear in z with slope -beta
  and zero intercept.

Materials: Al 6061 and basalt have alpha = beta, so an exchange is invisible in
their pressures; ice (alpha = 10, beta = 5) and a synthetic material with
alpha = 7, beta = 3 are where it shows.
"""
from dataclasses import replace

import numpy as np
import pytest

from paper_1604_03290_gb300 import workloads as wl


def _materials():
    return [wl.aluminium_6061(), wl.basalt(), wl.ice(),
            replace(wl.basalt(), name="alpha7beta3", alpha_T=7.0, beta_T=3.0)]


ETAS = (0.5, 0.6, 0.7, 0.8, 0.9, 0.95)


def _parts(mat, eta, u):
    rho = eta * mat.rho0
    z = 1.0 / eta - 1.0
    omega = 1.0 + u / (mat.E0 * eta * eta)
    return rho, z, omega


@pytest.mark.parametrize("mat", _materials(), ids=lambda m: m.name)
def test_alpha_factor_is_gaussian_in_z(orc, mat):
    zs, logs = [], []
    for eta in ETAS:
        rho, z, _ = _parts(mat, eta, 0)
        u1, u2 = 2.0 * mat.E_cv, 10.0 * mat.E_cv
        p1, p2 = orc.eos(mat, rho, u1)[0], orc.eos(mat, rho, u2)[0]
        w1, w2 = _parts(mat, eta, u1)[2], _parts(mat, eta, u2)[2]
        ratio = (p1 - p2 - mat.a_T * rho * (u1 - u2)) / (mat.b_T * rho * (u1 / w1 - u2 / w2))
        zs.append(z)
        logs.append(np.log(ratio))
    zs, logs = np.array(zs), np.array(logs)
    # least squares log(ratio) = c0 + c1 z + c2 z^2
    c0, c1, c2 = np.linalg.lstsq(np.vander(zs, 3, increasing=True), logs, rcond=None)[0]
    assert abs(c0) < 1e-9 and abs(c1) < 1e-8
    assert c2 == pytest.approx(-mat.alpha_T, rel=1e-9)


@pytest.mark.parametrize("mat", _materials(), ids=lambda m: m.name)
def test_beta_factor_is_exponential_in_z(orc, mat):
    zs, logs = [], []
    for eta in ETAS:
        rho, z, _ = _parts(mat, eta, 0)
        u = 2.0 * mat.E_cv
        w = _parts(mat, eta, u)[2]
        p = orc.eos(mat, rho, u)[0]
        cold = (p - mat.a_T * rho * u) * np.exp(mat.alpha_T * z * z) - mat.b_T * rho * u / w
        chi = eta - 1.0
        zs.append(z)
        logs.append(np.log(cold / (mat.A_T * chi)))
    zs, logs = np.array(zs), np.array(logs)
    c0, c1 = np.linalg.lstsq(np.vander(zs, 2, increasing=True), logs, rcond=None)[0]
    # the cold part is a difference of terms up to ~10x larger: a few 1e-13 of noise in the logs
    assert abs(c0) < 1e-7
    assert c1 == pytest.approx(-mat.beta_T, rel=1e-7)


def _numpy_expanded(mat, rho, u):
    """The expanded form of Eq. tillo2 written out independently with numpy."""
    eta = rho / mat.rho0
    chi = eta - 1.0
    x = mat.rho0 / rho - 1.0
    hot = mat.b_T * rho * u / (1.0 + u / (mat.E0 * eta ** 2))
    cold = mat.A_T * chi * np.exp(-mat.beta_T * x)
    return mat.a_T * rho * u + (hot + cold) * np.exp(-mat.alpha_T * x ** 2)


@pytest.mark.parametrize("mat", _materials(), ids=lambda m: m.name)
def test_expanded_pressure_at_interior_points(orc, mat):
    for eta in (0.5, 0.8, 0.95):
        for k in (1.0, 2.0, 10.0):
            rho, u = eta * mat.rho0, k * mat.E_cv
            p = orc.eos(mat, rho, u)[0]
            ref = _numpy_expanded(mat, rho, u)
            assert p == pytest.approx(ref, rel=1e-13, abs=1e-13 * mat.A_T)
            # a 1 % change of alpha or of beta moves p_e by far more than that tolerance
            for key in ("alpha_T", "beta_T"):
                moved = _numpy_expanded(replace(mat, **{key: getattr(mat, key) * 1.01}), rho, u)
                assert abs(moved - p) > 1e3 * 1e-13 * max(abs(p), mat.A_T * 1e-3), (key, eta, k)


def test_expanded_branch_is_taken_at_and_above_E_cv(orc):
    """u >= E_cv with rho < rho0 is pure p_e; just below E_cv the value is the
    interpolation, whose weight on p_c is (E_cv - u)/(E_cv - E_iv)."""
    mat = wl.ice()
    rho = 0.8 * mat.rho0
    pe = _numpy_expanded(mat, rho, mat.E_cv)
    assert orc.eos(mat, rho, mat.E_cv)[0] == pytest.approx(pe, rel=1e-13)
    u = 0.5 * (mat.E_iv + mat.E_cv)
    eta, chi = 0.8, -0.2
    pc = (mat.a_T + mat.b_T / (1 + u / (mat.E0 * eta * eta))) * rho * u + mat.A_T * chi + mat.B_T * chi * chi
    mid = 0.5 * (pc + _numpy_expanded(mat, rho, u))
    assert orc.eos(mat, rho, u)[0] == pytest.approx(mid, rel=1e-12, abs=1e-12 * mat.A_T)
