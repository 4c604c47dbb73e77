"""Host-side helpers on CPU: the material-parameter vector of the adjoint
(mu, Y0 and the bulk scale that moves K0, A_T and B_T together), the
penetration depth used as the adjoint's objective, and the autotuner's
candidate set (leaf size searched only without gravity)."""
from dataclasses import replace

import numpy as np
import torch

from paper_1604_03290_gb300 import autotune
from paper_1604_03290_gb300 import adjoint
from paper_1604_03290_gb300 import workloads as wl


def test_theta_round_trip_and_bulk_scaling():
    base = wl.ceres_pair(seed=4, n_each=50).materials
    mats = [base[0], replace(base[0], K0=3.0, A_T=0.0, B_T=0.0, mu=2.0, Y0=0.5)]
    th = adjoint.theta_of(mats)
    assert th.shape == (2, 3) and th.dtype == torch.float64
    np.testing.assert_array_equal(adjoint.theta_of(adjoint.materials_with(mats, th)).numpy(), th.numpy())
    new = th.clone()
    new[:, 0] *= 1.5
    new[:, 1] *= 0.5
    new[:, 2] *= 2.0
    out = adjoint.materials_with(mats, new)
    for m0, m1, t in zip(mats, out, new.numpy()):
        assert m1.mu == t[0] and m1.Y0 == t[1]
        # every bulk constant scales by the same factor (2), so their ratios and the EOS shape stay
        for f in ("K0", "A_T", "B_T"):
            np.testing.assert_allclose(getattr(m1, f), 2.0 * getattr(m0, f), rtol=1e-15)
        assert m1.rho0 == m0.rho0 and m1.eos == m0.eos


def test_penetration_depth_closed_form():
    x = torch.tensor([[0.0, 0.0, 0.0, 0.0], [0.0, 0.0, 0.0, 0.0], [-1.0, -3.0, 5.0, -2.0]], dtype=torch.float64)
    m = torch.tensor([1.0, 3.0, 7.0, 2.0], dtype=torch.float64)
    proj = torch.tensor([1.0, 1.0, 0.0, 1.0], dtype=torch.float64)
    d = adjoint.penetration_depth(x, m, proj, 0.5)
    np.testing.assert_allclose(d.numpy(), [0.5 - (-1.0 * 1 - 3.0 * 3 - 2.0 * 2) / 6.0])
    inst = torch.tensor([0, 0, 1, 1])
    d2 = adjoint.penetration_depth(x, m, proj, 0.5, inst_of_particle=inst, ninst=2)
    np.testing.assert_allclose(d2.numpy(), [0.5 - (-1.0 - 9.0) / 4.0, 0.5 + 2.0])
    # differentiable in the positions (the adjoint's seed)
    xr = x.clone().requires_grad_(True)
    adjoint.penetration_depth(xr, m, proj, 0.5).sum().backward()
    np.testing.assert_allclose(xr.grad[2].numpy(), -(m * proj / (m * proj).sum()).numpy())


def test_autotune_candidates():
    p = wl.Params(dim=3)
    c = autotune.candidates(p)
    assert len(c) == 3 * 4 * 4 * 2 and {x["leaf_size"] for x in c} == {8, 16, 32}
    g = autotune.candidates(replace(p, gravity=True, leaf_size=12))
    assert len(g) == 4 * 4 * 2 and {x["leaf_size"] for x in g} == {12}
    for x in c:
        assert 8 <= x["walk_leaf"] <= 1024 and 1 <= x["walk_blocks_per_sm"] <= 32 and x["pass_threads"] in (64, 128)
