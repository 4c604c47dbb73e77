"""Gradients of end-state quantities through predictor-corrector steps.

Reverse mode with step checkpointing: the forward pass keeps the state every
``every`` steps; the backward pass recomputes each segment from its
checkpoint and runs the hand-written adjoint of the update
(sph_pc_update_adjoint) and of the right-hand side (sph_rhs_adjoint) step by
step in reverse.  Partner lists and damage are those of the forward
evaluation (damage is held at its initial value: run with damage off), and
the time step is fixed.  The runner puts the particles in the tree order of
the initial state once (so that the partner gathers stay coherent) and keeps
that order for the whole trajectory; inputs, outputs and cotangents are in
the caller's order, permuted at the boundary.

``Rollout`` wraps this as a ``torch.autograd.Function`` of the initial
positions, velocities and the material parameters theta (nmat x 3: shear
modulus, yield stress, bulk modulus).
"""
from __future__ import annotations

from dataclasses import replace
from types import SimpleNamespace

import numpy as np
import torch

from . import sph
from . import workloads as wl


def materials_with(materials, theta):
    """Materials with mu, Y0 and the bulk modulus (K0, A_T, B_T scaled
    together, measured by the largest of them) taken from theta."""
    out = []
    th = theta.detach().cpu().double().numpy() if isinstance(theta, torch.Tensor) else np.asarray(theta, float)
    for m, t in zip(materials, th):
        kref = max(m.K0, m.A_T, m.B_T)
        s = t[2] / kref if kref > 0 else 1.0
        out.append(replace(m, mu=float(t[0]), Y0=float(t[1]), K0=m.K0 * s, A_T=m.A_T * s, B_T=m.B_T * s))
    return out


def theta_of(materials):
    return torch.tensor([[m.mu, m.Y0, max(m.K0, m.A_T, m.B_T)] for m in materials], dtype=torch.float64)


class Runner:
    """Fixed-dt predictor-corrector trajectory with checkpoints and its adjoint."""

    def __init__(self, ctx: sph.Context, template: wl.ParticleSet, params: wl.Params, dt, nsteps: int,
                 every: int = 10):
        assert not params.density_sum and not params.gravity and params.eps_s == 0.0, \
            "the adjoint covers continuity density without gravity or artificial stress"
        self.ctx = ctx
        self.params = params
        self.nsteps = int(nsteps)
        self.every = max(1, int(every))
        self.template = sph.DeviceState(template)
        # the tree order of the initial state: slot i holds particle order[i]
        sph.build_tree(ctx, self.template, params.leaf_size, params.max_depth, reorder=True)
        self.order = self.template.id.long()
        n = max(self.template.ninst, 1)
        self.dt = torch.as_tensor(np.broadcast_to(np.asarray(dt, np.float64), (n,)).copy(), device="cuda")
        self.d0 = sph.alloc_derivs(self.template)
        self.d1 = sph.alloc_derivs(self.template)
        self.fbar = sph.alloc_derivs(self.template)
        self.materials = None

    def _state(self, x0, v0):
        s = self.template.clone()
        s.x.copy_(x0[:, self.order])
        s.v.copy_(v0[:, self.order])
        return s

    def to_caller(self, t):
        """A (dim, n) tensor in the runner's order, back in the caller's."""
        out = torch.empty_like(t)
        out[:, self.order] = t
        return out

    def _step(self, q, qp):
        """q <- one step; qp receives the predicted state; d0 / d1 the derivatives."""
        ctx, P, M = self.ctx, self.params, self.materials
        sph.rhs(ctx, q, M, P, out=self.d0, check=False)
        sph.pc_update(ctx, q, self.d0, M, P, self.dt, 0.5, qp, check=False)
        sph.rhs(ctx, qp, M, P, out=self.d1, check=False)
        sph.pc_update(ctx, q, self.d1, M, P, self.dt, 1.0, q, check=False)

    def forward(self, x0, v0, theta):
        """The end state's positions and velocities (attributes x, v), in the
        caller's order, from x0, v0 in that order."""
        self.materials = materials_with(self.base_materials, theta)
        q = self._state(x0, v0)
        qp = q.clone()
        self.checkpoints = {0: q.clone()}
        for k in range(self.nsteps):
            self._step(q, qp)
            if (k + 1) % self.every == 0 and k + 1 < self.nsteps:
                self.checkpoints[k + 1] = q.clone()
        self.ctx.sync_status()
        return SimpleNamespace(x=self.to_caller(q.x), v=self.to_caller(q.v))

    def backward(self, xbar, vbar):
        """Cotangents of x0, v0 (attributes x, v, caller's order) and of the
        material parameters (ninst, nmat, 3) from those of the end state's
        positions and velocities (caller's order)."""
        ctx, P, M = self.ctx, self.params, self.materials
        nmat = len(M)
        ninst = max(self.template.ninst, 1)
        pbar = torch.zeros((ninst, nmat, 3), dtype=torch.float64, device="cuda")
        lam = self.template.zeros_like()
        lam.x.copy_(xbar[:, self.order])
        lam.v.copy_(vbar[:, self.order])
        lam_k = self.template.zeros_like()
        lam_p = self.template.zeros_like()
        qp = self.template.clone()
        starts = sorted(self.checkpoints)
        for si in range(len(starts) - 1, -1, -1):
            k0 = starts[si]
            k1 = starts[si + 1] if si + 1 < len(starts) else self.nsteps
            # recompute the segment's states
            states = [self.checkpoints[k0].clone()]
            for k in range(k0, k1 - 1):
                q = states[-1].clone()
                self._step(q, qp)
                states.append(q)
            for k in range(k1 - 1, k0 - 1, -1):
                q = states[k - k0]
                # forward pieces of step k
                sph.rhs(ctx, q, M, P, out=self.d0, check=False)
                sph.pc_update(ctx, q, self.d0, M, P, self.dt, 0.5, qp, check=False)
                sph.rhs(ctx, qp, M, P, out=self.d1, check=False)
                # corrector q' = Y(q + dt F(qp))
                for t in (lam_k, lam_p):
                    for name in ("x", "v", "rho", "u", "S"):
                        f = getattr(t, name)
                        if f is not None:
                            f.zero_()
                sph.pc_update_adjoint(ctx, q, self.d1, M, P, self.dt, 1.0, lam, lam_k, self.fbar, pbar, check=False)
                sph.rhs_adjoint(ctx, qp, M, P, self.fbar, lam_p, pbar, check=False)
                # predictor qp = Y(q + dt/2 F(q))
                sph.pc_update_adjoint(ctx, q, self.d0, M, P, self.dt, 0.5, lam_p, lam_k, self.fbar, pbar,
                                      check=False)
                sph.rhs_adjoint(ctx, q, M, P, self.fbar, lam_k, pbar, check=False)
                lam, lam_k = lam_k, lam
        ctx.sync_status()
        return SimpleNamespace(x=self.to_caller(lam.x), v=self.to_caller(lam.v)), pbar


class Rollout(torch.autograd.Function):
    """(x0, v0, theta) -> (x_N, v_N) through nsteps fixed-dt steps of the
    runner; backward = checkpointed hand-written adjoint."""

    @staticmethod
    def forward(fctx, x0, v0, theta, runner):
        q = runner.forward(x0, v0, theta)
        fctx.runner = runner
        return q.x.clone(), q.v.clone()

    @staticmethod
    def backward(fctx, gx, gv):
        runner = fctx.runner
        gx = torch.zeros_like(runner.template.x) if gx is None else gx.contiguous()
        gv = torch.zeros_like(runner.template.v) if gv is None else gv.contiguous()
        lam, pbar = runner.backward(gx, gv)
        return lam.x.clone(), lam.v.clone(), pbar.sum(0).to(torch.float64).cpu(), None


def rollout(runner: Runner, materials, x0, v0, theta):
    runner.base_materials = materials
    return Rollout.apply(x0, v0, theta, runner)


def penetration_depth(x, m, proj_mask, z_surface, inst_of_particle=None, ninst=1):
    """Mass-weighted mean depth of the projectile below z_surface along -z
    (per instance)."""
    z = x[-1]
    mp = m * proj_mask
    if ninst == 1:
        return (z_surface - (mp * z).sum() / mp.sum()).reshape(1)
    num = torch.zeros(ninst, dtype=x.dtype, device=x.device).index_add_(0, inst_of_particle, mp * z)
    den = torch.zeros(ninst, dtype=x.dtype, device=x.device).index_add_(0, inst_of_particle, mp)
    return z_surface - num / den
