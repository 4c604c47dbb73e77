"""sph_neighbours_static, the partner search that allocates no device memory,
against sph_neighbours with a context: identical CSR lists (integer work,
bit-exact) on calls in a row over different states that share the static
scratch, and clean capacity errors that leave the next call unaffected."""
import numpy as np
import pytest

from paper_1604_03290_gb300 import workloads as wl
from parity_util import flawed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_03290_gb300 import sph
    return sph


def _cases():
    solid = flawed(wl.measurement_1m(seed=4, n_side=20))                       # 3D, one body
    batch = flawed(wl.batched_impacts(seed=5, ninst=3, nmin=400, nmax=1500))   # 3D, three instances
    rings = wl.rings_2d(seed=3)                                        # 2D
    return [("solid", solid, 16, 21, 160), ("batch", batch, 16, 19, 256), ("rings", rings, 8, 21, 128)]


def _with_context(S, ps, leaf, depth, kmax):
    ctx = S.Context(ps.dim, ps.n, max_instances=max(ps.ninst, 1), max_neighbours=kmax)
    off, idx = S.neighbours(ctx, S.DeviceState(ps), leaf, depth)
    return off.cpu().numpy(), idx.cpu().numpy()


def test_static_lists_equal_context_lists_on_calls_in_a_row(S):
    cases = _cases()
    ref = {name: _with_context(S, ps, leaf, depth, kmax) for name, ps, leaf, depth, kmax in cases}
    # consecutive calls share the scratch: bigger, smaller, 2D, then the first again
    for name, ps, leaf, depth, kmax in cases + cases[:1]:
        off, idx = S.neighbours_static(S.DeviceState(ps), leaf, depth, kmax)
        ro, ri = ref[name]
        np.testing.assert_array_equal(off.cpu().numpy(), ro, err_msg=name)
        np.testing.assert_array_equal(idx.cpu().numpy(), ri, err_msg=name)
        assert ri.size > 5 * ps.n  # non-trivial lists


def test_static_rejects_sizes_beyond_the_scratch(S):
    big = flawed(wl.measurement_1m(seed=4, n_side=40))  # 64k particles: ~69 MB at 128 partners
    with pytest.raises(S.SphError) as e:
        S.neighbours_static(S.DeviceState(big), 16, 21, 128)
    assert e.value.status == S.SPH_ERR_CAPACITY
    assert "bytes of scratch" in str(e.value)
    name, ps, leaf, depth, kmax = _cases()[0]
    off, idx = S.neighbours_static(S.DeviceState(ps), leaf, depth, kmax)
    ro, ri = _with_context(S, ps, leaf, depth, kmax)
    np.testing.assert_array_equal(off.cpu().numpy(), ro)
    np.testing.assert_array_equal(idx.cpu().numpy(), ri)


def test_static_partner_overflow_is_reported_then_cleared(S):
    name, ps, leaf, depth, kmax = _cases()[0]
    ro, ri = _with_context(S, ps, leaf, depth, kmax)
    too_few = int(np.diff(ro).max()) - 1
    ds = S.DeviceState(ps)
    with pytest.raises(S.SphError) as e:
        S.neighbours_static(ds, leaf, depth, too_few)
    assert e.value.status == S.SPH_ERR_CAPACITY
    off, idx = S.neighbours_static(ds, leaf, depth, kmax)  # the error word of the last call is not carried over
    np.testing.assert_array_equal(off.cpu().numpy(), ro)
    np.testing.assert_array_equal(idx.cpu().numpy(), ri)


def test_static_calls_leave_device_free_memory_unchanged(S):
    """The promise itself: with the state and the outputs allocated up front
    (the caller's buffers), calls in a row change neither the device's free
    memory (cudaMemGetInfo) nor what torch's caching allocator holds.  The
    first call of the process may load the library's device code, array
    included, so one call runs before the readings start."""
    import ctypes as C

    import torch
    name, ps, leaf, depth, kmax = _cases()[0]
    ds = S.DeviceState(ps)
    S.neighbours_static(ds, leaf, depth, kmax)  # loads the module on this device
    cap = ps.n * kmax
    off = torch.zeros(ps.n + 1, dtype=torch.int64, device="cuda")
    idx = torch.zeros(cap, dtype=torch.int32, device="cuda")
    st = ds.struct()
    msg = C.create_string_buffer(512)
    lib = S.lib()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        r = lib.sph_neighbours_static(C.byref(st), leaf, depth, kmax, C.c_void_p(off.data_ptr()),
                                      C.c_void_p(idx.data_ptr()), cap, msg, len(msg), None)
        assert r == S.SPH_OK, msg.value
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_reserved() == reserved0
    ro, ri = _with_context(S, ps, leaf, depth, kmax)
    np.testing.assert_array_equal(off.cpu().numpy(), ro)
    np.testing.assert_array_equal(idx[: ri.size].cpu().numpy(), ri)
