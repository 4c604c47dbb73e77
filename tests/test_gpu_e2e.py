"""The end-to-end stepping of a state held in pinned host memory (bench.py's
host_steps: every step uploads all fields and downloads its result, with the
uploads of the next step overlapping the downloads) gives the same state,
bit for bit, as the same steps on a device-resident state; the device copy
is scrambled first, so only the uploads can make it right.  As in the bench,
one tree serves 4 steps and each one-step call continues the window of the
last, across the host round trip."""
import os
import sys
from dataclasses import replace

import numpy as np
import pytest

from paper_1604_03290_gb300 import workloads as wl
from parity_util import flawed

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_03290_gb300 import sph
    return sph


def test_host_steps_equal_device_steps(S):
    import torch
    sys.path.insert(0, ROOT)
    import bench
    ps = flawed(wl.measurement_1m(seed=11, n_side=30))
    prm = replace(ps.params, precision="mixed", tree_reuse=4)
    ctx = S.Context(3, ps.n, max_neighbours=128, leaf_size=prm.leaf_size)
    stream = torch.cuda.current_stream()
    ref = S.DeviceState(ps)
    S.step(ctx, ref, ps.materials, prm, 6, check=False)
    R = ref.to_numpy()
    ds = S.DeviceState(ps)
    host = {k: (None if v is None else v.detach().cpu().pin_memory()) for k, v in
            {"x": ds.x, "v": ds.v, "rho": ds.rho, "u": ds.u, "m": ds.m, "h": ds.h, "S": ds.S, "dmg": ds.dmg,
             "mat": ds.mat, "id": ds.id}.items()}
    for k in ("x", "v", "rho", "u", "m", "h", "S", "dmg"):
        getattr(ds, k).fill_(1.2345)
    bench.host_steps(S, ctx, ds, host, ps.materials, prm, 6, stream)
    torch.cuda.synchronize()
    ctx.sync_status()
    for k in ("x", "v", "rho", "u", "m", "h", "S", "dmg", "mat", "id"):
        np.testing.assert_array_equal(host[k].numpy(), R[k], err_msg=k)
