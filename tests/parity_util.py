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
