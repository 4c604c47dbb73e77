"""Helpers shared by the GPU parity tests: run both sides on one seeded input
and measure per-field errors against the oracle's own error scales."""
import numpy as np


def scaled_error(gpu, orc, scale):
    """max over particles of |gpu - orc| / scale (scale > 0)."""
    gpu = np.asarray(gpu, np.float64)
    orc = np.asarray(orc, np.float64)
    return float(np.max(np.abs(gpu - orc) / scale)) if gpu.size else 0.0


# Relative resolution of a kernel term evaluated in FP32 at the support edge,
# per unit of kappa = q/(1-q): about four roundings of q (2^-24 each) times the
# exponent 2 of (1-q)^2, with a factor two to spare -> 2^-19.  In FP64 the
# same with 2^-53 -> 2^-48.
EDGE = {"mixed": 2.0 ** -19, "fp64": 2.0 ** -48}


def field_scales(ps, o, prec="fp64", tol=1.0):
    """Per-particle error scales from the oracle's magnitude sums: sum_b
    |term_b| for each pair sum (for dS/dt the magnitude of the velocity
    gradient times (2 mu (1 + 1/D) + 4 max|S|)), plus the edge-conditioning
    sums sum_b |term_b| kappa_b weighted by EDGE[prec] / tol, so that
    |gpu - oracle| <= tol * scale means
    |gpu - oracle| <= tol * sum|term| + EDGE * sum|term| kappa."""
    n = ps.n
    tiny = 1e-300
    e = EDGE[prec] / tol
    mu = np.array([ps.materials[k].mu for k in ps.mat])
    smax = np.abs(ps.S).max(0) if ps.S is not None else np.zeros(n)
    gvs = 2 * mu * (1 + 1.0 / ps.dim) + 4 * smax
    sc = {
        "drho": o["mag_drho"] + e * o["mag1_drho"] + 1e-14 * max(o["mag_drho"].max(), tiny) + tiny,
        "dv": o["mag_dv"] + e * o["mag1_dv"] + np.sqrt((o["ag"] ** 2).sum(0)) +
              1e-14 * max(o["mag_dv"].max(), tiny) + tiny,
        "du": o["mag_du"] + e * o["mag1_du"] + 1e-14 * max(o["mag_du"].max(), tiny) + tiny,
        "dS": gvs * (o["mag_gradv"] + e * o["mag1_gradv"]) + tiny,
        "rho": o["mag_rho"] + e * o["mag1_rho"] + tiny,
        "dxdt": np.abs(ps.v).max() + tiny,
        "p": np.abs(o["p"]).max() + tiny,
        "cs": np.abs(o["cs"]).max() + tiny,
        "ddmg": np.abs(o["ddmg"]).max() + tiny,
    }
    sc["dS"] = sc["dS"] + 1e-14 * sc["dS"].max()
    return sc


def edge_share(ps, o, g, tol, prec, fields=("drho", "dv", "du", "dS")):
    """How much the edge-conditioning term of the tolerance is used: per field,
    the fraction of particles whose error exceeds tol times the bound without
    that term (they pass only because of it), and the largest ratio of error
    to that bound."""
    sc0 = field_scales(ps, {**o, **{k: np.zeros_like(v) for k, v in o.items() if k.startswith("mag1_")}}, prec, tol)
    out = {}
    for f in fields:
        if f == "dS" and ps.S is None:
            continue
        a, b = np.asarray(g[f], np.float64), np.asarray(o[f], np.float64)
        r = np.abs(a - b) / (tol * sc0[f])
        r = r.max(0) if r.ndim == 2 else r
        out[f] = (float((r > 1.0).mean()), float(r.max()))
    return out


def compare_rhs(ps, o, g, tol, fields=("drho", "dv", "du", "dS", "dxdt", "p", "cs"), report=None, prec="fp64"):
    sc = field_scales(ps, o, prec, tol)
    errs = {}
    for f in fields:
        if f == "dS" and ps.S is None:
            continue
        a, b = np.asarray(g[f]), np.asarray(o[f])
        s = sc[f]
        if a.ndim == 2:
            errs[f] = max(scaled_error(a[k], b[k], s) for k in range(a.shape[0]))
        else:
            errs[f] = scaled_error(a, b, s)
    if report is not None:
        report.update(errs)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, "fields over tolerance %g: %s (all: %s)" % (tol, bad, errs)
    return errs


def check_damage(ps, o, g, prec, tol, report=None):
    """Activated flaws and damage growth (Sects. 2.7, 3.2) against the oracle.

    FP64: n_act equal everywhere.  Mixed: the constitutive update runs in
    FP32, so the local strain eps = sigma_max / ((1 - d) E) carries an error of
    its own; a count may differ only where every threshold counted by one side
    and not the other lies within that error of the oracle's eps:
        |eps_j - eps| <= (|p_gpu - p| + 2^-18 ((1 - d) |S|_F + |p|)) / ((1 - d) E) + 2^-20 |eps|,
    i.e. the particle's own pressure difference (bounded by the pressure test)
    plus 64 FP32 roundings of the stress magnitude for the eigen-solve and 16
    of eps itself.  Where the counts agree, d(d^1/3)/dt matches to the field
    tolerance; where they differ it must be the growth of the GPU's count,
    n_act c_g / h (R16, R17) while d < n_act / n_tot, else 0."""
    if ps.dmg is None:
        return
    n_g, n_o = np.asarray(g["n_act"]), np.asarray(o["n_act"])
    same = n_g == n_o
    scale = np.abs(o["ddmg"]).max() + 1e-300
    if prec == "fp64":
        assert same.all(), "n_act differs on %d particles" % (~same).sum()
    bad = np.flatnonzero(~same)
    u32 = 2.0 ** -24
    mats = ps.materials
    off, thr = np.asarray(ps.flaw_off), np.asarray(ps.flaw_eps, np.float64)
    ids = np.asarray(ps.id)
    expect = np.array(g["ddmg"], np.float64, copy=True)
    for a in bad:
        M = mats[int(ps.mat[a])]
        dd = float(ps.dmg[a]) ** 3
        E = 9 * M.K0 * M.mu / (3 * M.K0 + M.mu)
        den = (1 - dd) * E
        Sf = float(np.sqrt((ps.S[:, a] ** 2).sum() + (ps.S[ps.dim:, a] ** 2).sum())) if ps.S is not None else 0.0
        delta = (abs(g["p"][a] - o["p"][a]) + 64 * u32 * ((1 - dd) * Sf + abs(o["p"][a]))) / den + \
            16 * u32 * abs(o["eps_t"][a])
        t = thr[off[ids[a]]:off[ids[a] + 1]]
        lo, hi = min(n_g[a], n_o[a]), max(n_g[a], n_o[a])
        e = max(o["eps_t"][a], 0.0)
        assert np.all(np.abs(t[lo:hi] - e) <= delta), \
            "particle %d: n_act %d vs %d, eps %.9g, thresholds %s, bound %.3g" % (a, n_g[a], n_o[a], e, t[lo:hi], delta)
        ntot = len(t)
        rate = 0.4 * np.sqrt((M.K0 + 4.0 / 3.0 * (1 - dd) * M.mu) / ps.rho[a]) / ps.h[a]
        expect[a] = n_g[a] * rate if (n_g[a] > 0 and dd < n_g[a] / ntot) else 0.0
    err_same = float(np.abs(g["ddmg"] - o["ddmg"])[same].max() / scale) if same.any() else 0.0
    err_flip = float(np.abs(g["ddmg"] - expect)[bad].max() / scale) if bad.size else 0.0
    if report is not None:
        report.update({"n_act_flips": int(bad.size), "ddmg_same": err_same, "ddmg_flipped": err_flip})
    assert err_same <= 10 * tol, err_same
    assert err_flip <= 10 * tol, err_flip


def flawed(ps):
    """The particle set with its Weibull flaws drawn by the oracle (orc_flaws,
    Sect. 3.2) from its flaw_seed, so that both sides of a comparison read the
    same pinned flaws; returns ps."""
    import oracle
    return oracle.ensure_flaws(ps)
