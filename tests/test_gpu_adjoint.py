"""Hand-written adjoint: dot-product test of the right-hand-side adjoint against
central differences, and gradients of penetration depth through checkpointed
predictor-corrector steps against FP64 central finite differences of the GPU
forward and of the CPU oracle (target 1e-4 relative)."""
from dataclasses import replace

import numpy as np
import pytest

from paper_1604_03290_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_03290_gb300 import sph
    return sph


def _solid(seed=21, n_side=10):
    ps = wl.measurement_1m(seed=seed, n_side=n_side, damage=False)
    rng = np.random.default_rng(seed)
    ps.u = rng.uniform(0.0, 6e6, ps.n)          # compressed, cold and mixed Tillotson branches
    ps.S = rng.normal(0.0, 0.4 * ps.materials[0].Y0, (6, ps.n))  # some particles yield
    ps.params = replace(ps.params, alpha=1.0, beta=2.0, xsph=0.5, precision="fp64")
    return ps


def _dot(a, b):
    return float(sum((x * y).sum() for x, y in zip(a, b)))


def test_rhs_adjoint_dot_product(S):
    import torch
    ps = _solid()
    prm = ps.params
    ctx = S.Context(3, ps.n, max_neighbours=160)
    rng = np.random.default_rng(5)
    ds = S.DeviceState(ps)
    n = ps.n
    dx = 0.1 / 100
    # random output cotangents
    W = {"dxdt": rng.normal(size=(3, n)) * 1e-3, "dv": rng.normal(size=(3, n)) * 1e-6, "drho": rng.normal(size=n),
         "du": rng.normal(size=n) * 1e-6, "dS": rng.normal(size=(6, n)) * 1e-9}
    Wt = {k: torch.as_tensor(v, device="cuda") for k, v in W.items()}
    dbar = S.alloc_derivs(ds)
    for k, v in Wt.items():
        dbar[k].copy_(v)
    sbar = ds.zeros_like()
    pbar = torch.zeros((1, 1, 3), dtype=torch.float64, device="cuda")
    S.rhs_adjoint(ctx, ds, ps.materials, prm, dbar, sbar, pbar)
    adj = sbar.to_numpy()
    # random state direction
    D = {"x": rng.normal(size=(3, n)) * 1e-2 * dx, "v": rng.normal(size=(3, n)), "rho": rng.normal(size=n) * 2.7,
         "u": rng.normal(size=n) * 1e4, "S": rng.normal(size=(6, n)) * 1e5}

    def F(sign, eps, mats=None):
        q = ps.copy()
        for k, v in D.items():
            setattr(q, k, getattr(ps, k) + sign * eps * v)
        out = S.rhs(ctx, S.DeviceState(q), mats or ps.materials, prm)
        return [out[k].cpu().numpy() for k in ("dxdt", "dv", "drho", "du", "dS")]

    eps = 1e-3
    Fp, Fm = F(1, eps), F(-1, eps)
    Wl = [W[k] for k in ("dxdt", "dv", "drho", "du", "dS")]
    lhs = _dot(Wl, [(a - b) / (2 * eps) for a, b in zip(Fp, Fm)])
    rhs = _dot([adj[k] for k in D], [D[k] for k in D])
    mag = _dot([np.abs(w) for w in Wl], [np.abs(a - b) / (2 * eps) for a, b in zip(Fp, Fm)])
    assert abs(lhs - rhs) <= 1e-6 * mag, (lhs, rhs, mag)
    # parameter directions: mu, Y0, K
    m0 = ps.materials[0]
    kref = max(m0.K0, m0.A_T, m0.B_T)
    for j, (name, val) in enumerate((("mu", m0.mu), ("Y0", m0.Y0), ("K", kref))):
        e = 1e-5 * val

        def mats(sign):
            if name == "K":
                s = (kref + sign * e) / kref
                return [replace(m0, K0=m0.K0 * s, A_T=m0.A_T * s, B_T=m0.B_T * s)]
            return [replace(m0, **{name: val + sign * e})]

        D_save = dict(D)
        D.clear()
        Fp, Fm = F(1, 0.0, mats(1)), F(-1, 0.0, mats(-1))
        D.update(D_save)
        lhs = _dot(Wl, [(a - b) / (2 * e) for a, b in zip(Fp, Fm)])
        mag = _dot([np.abs(w) for w in Wl], [np.abs(a - b) / (2 * e) for a, b in zip(Fp, Fm)])
        got = float(pbar[0, 0, j].item())
        assert abs(lhs - got) <= 1e-5 * mag + 1e-30, (name, lhs, got, mag)


def _batch(ninst=2):
    ps = wl.batched_impacts(seed=7, ninst=ninst, nmin=300, nmax=700, with_flaws=False)
    mat = replace(ps.materials[0], damage=False)
    ps.materials = [mat]
    ps.dmg = None
    ps.params = replace(ps.params, max_depth=18, alpha=1.0, beta=2.0, precision="fp64")
    return ps


def _depth_numpy(x, m, proj, inst_off):
    out = []
    for i in range(len(inst_off) - 1):
        sl = slice(inst_off[i], inst_off[i + 1])
        mp = m[sl] * proj[sl]
        out.append(-(mp * x[2][sl]).sum() / mp.sum())
    return np.array(out)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_step_adjoint_matches_finite_differences(S, orc, prec):
    # mixed: the rollout and its adjoint in mixed precision, against the oracle's
    # FP64 finite differences (finite differences of the mixed trajectory itself
    # would be FP32 rounding noise)
    import torch
    from paper_1604_03290_gb300 import adjoint
    ps = _batch()
    nsteps, every = 12, 5
    cmax = np.sqrt(ps.materials[0].A_T / ps.materials[0].rho0)
    dt = 0.25 * ps.h.min() / (cmax + 6000.0)
    prm = replace(ps.params, dt_fixed=dt, precision=prec)
    ctx = S.Context(3, ps.n, max_instances=4, max_neighbours=160)
    runner = adjoint.Runner(ctx, ps, prm, dt, nsteps, every=every)
    proj = (ps.v[2] < 0).astype(float)
    inst = np.repeat(np.arange(ps.ninst), np.diff(ps.inst_off))
    x0 = torch.as_tensor(ps.x, device="cuda")
    v0 = torch.as_tensor(ps.v, device="cuda")
    m = torch.as_tensor(ps.m, device="cuda")
    projt = torch.as_tensor(proj, device="cuda")
    instt = torch.as_tensor(inst, device="cuda")
    theta = adjoint.theta_of(ps.materials).requires_grad_(True)
    v0r = v0.clone().requires_grad_(True)
    xN, vN = adjoint.rollout(runner, ps.materials, x0, v0r, theta)
    J = adjoint.penetration_depth(xN, m, projt, 0.0, instt, ps.ninst)
    J.sum().backward()
    gv = v0r.grad.cpu().numpy()
    gth = theta.grad.numpy()[0]
    # dJ/dV0 per instance: the projectile moves along -z at speed V0
    g_speed = np.array([-(gv[2] * proj)[inst == i].sum() for i in range(ps.ninst)])

    def J_gpu(v=None, mats=None):
        runner.base_materials = mats or ps.materials
        q = runner.forward(x0, torch.as_tensor(v if v is not None else ps.v, device="cuda"),
                           adjoint.theta_of(runner.base_materials))
        return _depth_numpy(q.x.cpu().numpy(), ps.m, proj, ps.inst_off)

    def J_orc(v=None, mats=None):
        q = ps.copy()
        if v is not None:
            q.v = v
        st, _ = orc.step(q, mats or ps.materials, replace(prm, precision="fp64"), nsteps)
        return _depth_numpy(st["x"], ps.m, proj, ps.inst_off)

    fp64 = prec == "fp64"

    fd_gpu, fd_orc = [], []
    for i in range(ps.ninst):
        dv = np.zeros_like(ps.v)
        sel = (inst == i) & (proj > 0)
        dV = 1e-6 * np.abs(ps.v[2][sel]).max()  # steps small enough not to cross branch switches
        dv[2][sel] = -dV  # increase the speed
        if fp64:
            fd_gpu.append((J_gpu(ps.v + dv)[i] - J_gpu(ps.v - dv)[i]) / (2 * dV))
        fd_orc.append((J_orc(ps.v + dv)[i] - J_orc(ps.v - dv)[i]) / (2 * dV))
    print("dJ/dV0", prec, g_speed, fd_gpu, fd_orc)
    if fp64:
        np.testing.assert_allclose(g_speed, fd_gpu, rtol=1e-4)
    np.testing.assert_allclose(g_speed, fd_orc, rtol=1e-4)
    m0 = ps.materials[0]
    kref = max(m0.K0, m0.A_T, m0.B_T)
    for j, (name, val) in enumerate((("mu", m0.mu), ("Y0", m0.Y0), ("K", kref))):
        # J is piecewise smooth (yield, EOS-branch and viscosity switches):
        # 1e-6 relative steps stay on one side of the switches
        e = 1e-6 * val

        def mats(sign):
            if name == "K":
                s = (kref + sign * e) / kref
                return [replace(m0, K0=m0.K0 * s, A_T=m0.A_T * s, B_T=m0.B_T * s)]
            return [replace(m0, **{name: val + sign * e})]

        fdo = (J_orc(mats=mats(1)).sum() - J_orc(mats=mats(-1)).sum()) / (2 * e)
        # sensitivities below 1e-8 of |J| / theta count as zero
        floor = 1e-8 * float(J.detach().abs().sum()) / val
        print(name, prec, gth[j], fdo)
        if fp64:
            fdg = (J_gpu(mats=mats(1)).sum() - J_gpu(mats=mats(-1)).sum()) / (2 * e)
            assert abs(gth[j] - fdg) <= 1e-4 * abs(fdg) + floor, (name, gth[j], fdg)
        assert abs(gth[j] - fdo) <= 1e-4 * abs(fdo) + floor, (name, gth[j], fdo)


def test_rhs_adjoint_mixed_matches_fp64(S):
    # the mixed form (FP32 pair terms in code units, FP64 constitutive reverse)
    # against the FP64 adjoint on the same state and output cotangents
    import torch
    ps = _solid()
    ctx = S.Context(3, ps.n, max_neighbours=160)
    rng = np.random.default_rng(6)
    n = ps.n
    W = {"dxdt": rng.normal(size=(3, n)) * 1e-3, "dv": rng.normal(size=(3, n)) * 1e-6, "drho": rng.normal(size=n),
         "du": rng.normal(size=n) * 1e-6, "dS": rng.normal(size=(6, n)) * 1e-9}
    res = {}
    for prec in ("fp64", "mixed"):
        ds = S.DeviceState(ps)
        dbar = S.alloc_derivs(ds)
        for k, v in W.items():
            dbar[k].copy_(torch.as_tensor(v, device="cuda"))
        sbar = ds.zeros_like()
        pbar = torch.zeros((1, 1, 3), dtype=torch.float64, device="cuda")
        S.rhs_adjoint(ctx, ds, ps.materials, replace(ps.params, precision=prec), dbar, sbar, pbar)
        res[prec] = (sbar.to_numpy(), pbar.cpu().numpy()[0, 0])
    a, b = res["fp64"][0], res["mixed"][0]
    for k in ("x", "v", "rho", "u", "S"):
        scale = np.abs(a[k]).max()
        err = np.abs(b[k] - a[k]).max() / scale
        print("mixed adjoint", k, err)
        assert err <= 1e-4, (k, err)
    np.testing.assert_allclose(res["mixed"][1], res["fp64"][1], rtol=1e-4)
