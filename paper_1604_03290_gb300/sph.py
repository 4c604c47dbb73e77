"""Thin ctypes binding of ``libsph.so`` (include/sph.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch provides device memory and streams.  If the library or a
CUDA device is missing, the calls raise; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import workloads as wl

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsph.so")
_lock = threading.Lock()
_lib = None

SPH_OK, SPH_ERR_INVALID, SPH_ERR_CAPACITY, SPH_ERR_NONFINITE, SPH_ERR_TIMEOUT, SPH_ERR_CUDA = range(6)
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "CAPACITY", 3: "NONFINITE", 4: "TIMEOUT", 5: "CUDA"}
EOS = {"linear": 0, "murnaghan": 1, "tillotson": 2, "isothermal": 3}
PRECISION = {"fp64": 0, "mixed": 1}
PHASES = ("tree", "reorder", "partners", "density", "passA", "passB", "gravity", "integrate", "flaw_draws",
          "flaw_fill", "fof_links", "refine")
COUNTERS = ("grav_nodes", "grav_terms", "grav_visits", "walk_tests", "walk_partners")


class SphError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class Material(C.Structure):
    _fields_ = [("eos", C.c_int32), ("strength", C.c_int32), ("damage", C.c_int32), ("pad", C.c_int32),
                ("rho0", C.c_double), ("cs", C.c_double), ("K0", C.c_double), ("n_M", C.c_double),
                ("A_T", C.c_double), ("B_T", C.c_double), ("E0", C.c_double), ("E_iv", C.c_double),
                ("E_cv", C.c_double), ("a_T", C.c_double), ("b_T", C.c_double), ("alpha_T", C.c_double),
                ("beta_T", C.c_double), ("rho_cut", C.c_double), ("mu", C.c_double), ("Y0", C.c_double)]


class Params(C.Structure):
    _fields_ = [("dim", C.c_int32), ("density_sum", C.c_int32), ("consistency", C.c_int32),
                ("gravity", C.c_int32), ("leaf_size", C.c_int32), ("max_depth", C.c_int32),
                ("precision", C.c_int32), ("check", C.c_int32),
                ("alpha", C.c_double), ("beta", C.c_double), ("eps_v", C.c_double),
                ("eps_s", C.c_double), ("n_as", C.c_double), ("dmpd", C.c_double), ("xsph", C.c_double),
                ("G", C.c_double), ("theta", C.c_double), ("eps_grav", C.c_double),
                ("c_courant", C.c_double), ("c_accel", C.c_double), ("c_quantity", C.c_double),
                ("u_floor", C.c_double), ("S_floor", C.c_double), ("dmg_floor", C.c_double),
                ("dt_max", C.c_double), ("dt_fixed", C.c_double), ("n_des", C.c_double),
                ("h_tol", C.c_int32), ("h_iter", C.c_int32), ("tree_reuse", C.c_int32),
                ("tree_continue", C.c_int32)]


_vp = C.c_void_p


class State(C.Structure):
    _fields_ = [("dim", C.c_int32), ("ninst", C.c_int32), ("n", C.c_int64), ("x", _vp * 3), ("v", _vp * 3),
                ("rho", _vp), ("u", _vp), ("m", _vp), ("h", _vp), ("S", _vp), ("dmg", _vp), ("mat", _vp),
                ("id", _vp), ("flaw_off", _vp), ("flaw_eps", _vp), ("inst_off", _vp)]


class Tuning(C.Structure):
    _fields_ = [("walk_leaf", C.c_int32), ("walk_blocks_per_sm", C.c_int32), ("pass_threads", C.c_int32),
                ("walk_every_eval", C.c_int32), ("iter_cap", C.c_int32), ("plain_forms", C.c_int32)]


class Derivs(C.Structure):
    _fields_ = [("dx", _vp * 3), ("dv", _vp * 3), ("drho", _vp), ("du", _vp), ("dS", _vp), ("ddmg", _vp),
                ("cs", _vp), ("p", _vp), ("n_act", _vp), ("nnb", _vp)]


def lib():
    """Loads libsph.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build as _build
            _build.build()
            L = C.CDLL(LIB_PATH)
            L.sph_create.argtypes = [C.POINTER(_vp), C.c_int32, C.c_int64, C.c_int32, C.c_int32, C.c_int32, _vp]
            L.sph_destroy.argtypes = [_vp]
            L.sph_destroy.restype = None
            L.sph_last_error.argtypes = [_vp]
            L.sph_last_error.restype = C.c_char_p
            L.sph_sync_status.argtypes = [_vp, _vp]
            L.sph_ctx_bytes.argtypes = [_vp]
            L.sph_ctx_bytes.restype = C.c_int64
            L.sph_build_tree.argtypes = [_vp, C.POINTER(State), C.c_int32, C.c_int32, C.c_int32, _vp, _vp]
            L.sph_tree_nodes.argtypes = [_vp, C.c_int64, _vp, _vp, _vp, _vp, _vp, C.POINTER(C.c_int64), _vp]
            L.sph_neighbours.argtypes = [_vp, C.POINTER(State), C.c_int32, C.c_int32, _vp, _vp, C.c_int64, _vp]
            L.sph_rhs.argtypes = [_vp, C.POINTER(State), C.POINTER(Material), C.c_int32, C.POINTER(Params),
                                  C.POINTER(Derivs), _vp]
            L.sph_gravity.argtypes = [_vp, C.POINTER(State), C.POINTER(Params), _vp, _vp, _vp, _vp]
            L.sph_step_rk3.argtypes = [_vp, C.POINTER(State), C.POINTER(Material), C.c_int32, C.POINTER(Params),
                                       C.c_double, _vp, _vp, C.c_int32, _vp, _vp, _vp]
            L.sph_adapt_h.argtypes = [_vp, C.POINTER(State), C.c_int32, C.c_int32, C.c_double, C.c_int32,
                                      C.c_int32, _vp, C.POINTER(C.c_int32), _vp]
            L.sph_neighbours_static.argtypes = [C.POINTER(State), C.c_int32, C.c_int32, C.c_int32, _vp, _vp,
                                                C.c_int64, C.c_char_p, C.c_int32, _vp]
            L.sph_step.argtypes = [_vp, C.POINTER(State), C.POINTER(Material), C.c_int32, C.POINTER(Params), _vp,
                                   C.c_int32, _vp]
            L.sph_flaws.argtypes = [_vp, C.POINTER(State), C.POINTER(Material), C.c_int32, _vp, _vp, C.c_uint64,
                                    _vp, _vp, C.c_int64, C.POINTER(C.c_int64), _vp]
            L.sph_fragments.argtypes = [_vp, C.POINTER(State), _vp, C.c_double, C.c_double, C.c_int32, C.c_int32,
                                        C.c_int32, _vp, _vp, _vp, C.c_int64, C.POINTER(C.c_int64), _vp]
            L.sph_measure_fma_peak.argtypes = [C.c_int32, C.POINTER(C.c_double)]
            L.sph_profile_enable.argtypes = [_vp, C.c_int32]
            L.sph_profile_read.argtypes = [_vp, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.c_int32]
            L.sph_profile_counters.argtypes = [_vp, C.POINTER(C.c_int64), C.c_int32, _vp]
            L.sph_rhs_adjoint.argtypes = [_vp, C.POINTER(State), C.POINTER(Material), C.c_int32, C.POINTER(Params),
                                          C.POINTER(Derivs), C.POINTER(State), _vp, _vp]
            L.sph_pc_update.argtypes = [_vp, C.POINTER(State), C.POINTER(Derivs), C.POINTER(Material), C.c_int32,
                                        C.POINTER(Params), _vp, C.c_double, C.POINTER(State), _vp]
            L.sph_pc_update_adjoint.argtypes = [_vp, C.POINTER(State), C.POINTER(Derivs), C.POINTER(Material),
                                                C.c_int32, C.POINTER(Params), _vp, C.c_double, C.POINTER(State),
                                                C.POINTER(State), C.POINTER(Derivs), _vp, _vp]
            L.sph_get_tuning.argtypes = [_vp, C.POINTER(Tuning)]
            L.sph_set_tuning.argtypes = [_vp, C.POINTER(Tuning)]
            L.sph_launch_count.argtypes = []
            L.sph_launch_count.restype = C.c_int64
            for f in ("sph_create", "sph_sync_status", "sph_build_tree", "sph_tree_nodes", "sph_neighbours",
                      "sph_neighbours_static", "sph_adapt_h", "sph_step_rk3", "sph_flaws", "sph_fragments",
                      "sph_rhs", "sph_gravity", "sph_step", "sph_measure_fma_peak", "sph_profile_enable",
                      "sph_profile_read", "sph_profile_counters", "sph_get_tuning", "sph_set_tuning", "sph_rhs_adjoint", "sph_pc_update",
                      "sph_pc_update_adjoint"):
                getattr(L, f).restype = C.c_int
            _lib = L
    return _lib


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("the SPH library needs a CUDA device; there is no CPU fallback")


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else t.data_ptr()


def _stream(stream):
    return (stream if stream is not None else torch.cuda.current_stream()).cuda_stream


def material_struct(m: wl.Material) -> Material:
    s = Material()
    s.eos = EOS[m.eos]
    s.strength = int(m.strength)
    s.damage = int(m.damage)
    for k in ("rho0", "cs", "K0", "n_M", "A_T", "B_T", "E0", "E_iv", "E_cv", "a_T", "b_T", "alpha_T",
              "beta_T", "rho_cut", "mu", "Y0"):
        setattr(s, k, float(getattr(m, k)))
    return s


def params_struct(p: wl.Params, check: bool = True, cont: bool = False) -> Params:
    s = Params()
    ints = ("dim", "density_sum", "consistency", "gravity", "leaf_size", "max_depth", "h_tol", "h_iter",
            "tree_reuse")
    for k, _ in Params._fields_:
        if k == "precision":
            s.precision = PRECISION[p.precision]
        elif k == "check":
            s.check = int(check)
        elif k == "tree_continue":
            s.tree_continue = int(cont)
        else:
            v = getattr(p, k)
            setattr(s, k, int(v) if k in ints else float(v))
    return s


def materials_array(mats):
    arr = (Material * len(mats))()
    for i, m in enumerate(mats):
        arr[i] = material_struct(m)
    return arr


class Context:
    """Owns the library context (all scratch, sized once)."""

    def __init__(self, dim: int, max_particles: int, max_instances: int = 1, max_neighbours: int = 128,
                 leaf_size: int = 16):
        _require_cuda()
        self._lib = lib()
        h = _vp()
        st = lib().sph_create(C.byref(h), int(dim), int(max_particles), int(max_instances), int(max_neighbours),
                              int(leaf_size), None)
        if st != SPH_OK:
            raise SphError(st, "sph_create failed")
        self.h = h
        self.dim = dim
        self.max_particles = max_particles
        self.max_neighbours = max_neighbours

    def close(self):
        if getattr(self, "h", None):
            self._lib.sph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def bytes(self):
        return int(self._lib.sph_ctx_bytes(self.h))

    def check(self, status, what):
        if status != SPH_OK:
            raise SphError(status, "%s: %s" % (what, self._lib.sph_last_error(self.h).decode()))

    def sync_status(self, stream=None):
        self.check(self._lib.sph_sync_status(self.h, _stream(stream)), "device status")

    def get_tuning(self) -> dict:
        t = Tuning()
        self.check(self._lib.sph_get_tuning(self.h, C.byref(t)), "sph_get_tuning")
        return {"walk_leaf": t.walk_leaf, "walk_blocks_per_sm": t.walk_blocks_per_sm, "pass_threads": t.pass_threads,
                "walk_every_eval": t.walk_every_eval, "iter_cap": t.iter_cap, "plain_forms": t.plain_forms}

    def set_tuning(self, **kw):
        cur = self.get_tuning()
        cur.update(kw)
        t = Tuning(cur["walk_leaf"], cur["walk_blocks_per_sm"], cur["pass_threads"], int(cur["walk_every_eval"]),
                   int(cur["iter_cap"]), int(cur["plain_forms"]))
        self.check(self._lib.sph_set_tuning(self.h, C.byref(t)), "sph_set_tuning")

    def profile(self, on=True):
        self.check(self._lib.sph_profile_enable(self.h, int(on)), "sph_profile_enable")

    def profile_counters(self, stream=None):
        """Interaction counters of the walks since profiling began or the last
        read (sph_profile_counters), then reset."""
        out = (C.c_int64 * len(COUNTERS))()
        self.check(self._lib.sph_profile_counters(self.h, out, len(COUNTERS), _stream(stream)),
                   "sph_profile_counters")
        return {k: int(out[i]) for i, k in enumerate(COUNTERS)}

    def profile_read(self):
        ms = (C.c_double * len(PHASES))()
        calls = (C.c_int32 * len(PHASES))()
        self.check(self._lib.sph_profile_read(self.h, ms, calls, len(PHASES)), "sph_profile_read")
        return {p: (ms[i], calls[i]) for i, p in enumerate(PHASES)}


class DeviceState:
    """Particle state in device memory (torch tensors) plus its sph_state view."""

    def __init__(self, ps: wl.ParticleSet, device="cuda"):
        _require_cuda()
        if ps.flaw_off is None and getattr(ps, "flaw_seed", None) is not None:
            raise ValueError("the particle set's Weibull flaws are not drawn yet: fill_flaws(ctx, ps) draws them "
                             "on the device from ps.flaw_seed")
        f64 = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64,
                                                                device=device).contiguous()
        self.dim = ps.dim
        self.n = ps.n
        self.x = f64(ps.x)
        self.v = f64(ps.v)
        self.rho = f64(ps.rho)
        self.u = f64(ps.u)
        self.m = f64(ps.m)
        self.h = f64(ps.h)
        self.S = f64(ps.S)
        self.dmg = f64(ps.dmg)
        self.mat = torch.as_tensor(np.asarray(ps.mat, np.int32), device=device)
        self.id = torch.as_tensor(np.asarray(ps.id, np.int32), device=device)
        self.flaw_off = None if ps.flaw_off is None else torch.as_tensor(np.asarray(ps.flaw_off, np.int64),
                                                                         device=device)
        self.flaw_eps = None if ps.flaw_eps is None else torch.as_tensor(np.asarray(ps.flaw_eps, np.float32),
                                                                         device=device)
        self.inst_off = None if ps.inst_off is None else torch.as_tensor(np.asarray(ps.inst_off, np.int64),
                                                                         device=device)
        self.ninst = ps.ninst

    def struct(self) -> State:
        s = State()
        s.dim = self.dim
        s.ninst = self.ninst
        s.n = self.n
        for k in range(3):
            s.x[k] = _ptr(self.x[k]) if k < self.dim else None
            s.v[k] = _ptr(self.v[k]) if k < self.dim else None
        s.rho, s.u, s.m, s.h = _ptr(self.rho), _ptr(self.u), _ptr(self.m), _ptr(self.h)
        s.S, s.dmg = _ptr(self.S), _ptr(self.dmg)
        s.mat, s.id = _ptr(self.mat), _ptr(self.id)
        s.flaw_off, s.flaw_eps = _ptr(self.flaw_off), _ptr(self.flaw_eps)
        s.inst_off = _ptr(self.inst_off) if self.ninst > 1 else None
        return s

    def clone(self):
        """A copy of the evolving fields (x, v, rho, u, S, dmg) sharing the constant ones."""
        c = object.__new__(DeviceState)
        c.__dict__.update(self.__dict__)
        for k in ("x", "v", "rho", "u", "S", "dmg"):
            t = getattr(self, k)
            setattr(c, k, None if t is None else t.clone())
        return c

    def copy_from(self, other):
        for k in ("x", "v", "rho", "u", "S", "dmg"):
            t = getattr(self, k)
            if t is not None:
                t.copy_(getattr(other, k))

    def zeros_like(self):
        """Same layout, evolving fields set to zero (a cotangent container)."""
        c = self.clone()
        for k in ("x", "v", "rho", "u", "S", "dmg"):
            t = getattr(c, k)
            if t is not None:
                t.zero_()
        return c

    def to_numpy(self):
        g = lambda t: None if t is None else t.detach().cpu().numpy()
        return {"x": g(self.x), "v": g(self.v), "rho": g(self.rho), "u": g(self.u), "S": g(self.S),
                "dmg": g(self.dmg), "id": g(self.id), "m": g(self.m), "h": g(self.h), "mat": g(self.mat)}


def alloc_derivs(ds: DeviceState, device="cuda"):
    n, dim = ds.n, ds.dim
    ns = 6 if dim == 3 else 3
    z = lambda *s: torch.zeros(*s, dtype=torch.float64, device=device)
    out = {"dxdt": z(dim, n), "dv": z(dim, n), "drho": z(n), "du": z(n), "dS": z(ns, n), "ddmg": z(n),
           "cs": z(n), "p": z(n), "n_act": torch.zeros(n, dtype=torch.int32, device=device),
           "nnb": torch.zeros(n, dtype=torch.int32, device=device)}
    return out


def derivs_struct(out) -> Derivs:
    d = Derivs()
    dim = out["dv"].shape[0]
    for k in range(3):
        d.dx[k] = _ptr(out["dxdt"][k]) if k < dim else None
        d.dv[k] = _ptr(out["dv"][k]) if k < dim else None
    d.drho, d.du, d.dS, d.ddmg = _ptr(out["drho"]), _ptr(out["du"]), _ptr(out["dS"]), _ptr(out["ddmg"])
    d.cs, d.p, d.n_act, d.nnb = _ptr(out["cs"]), _ptr(out["p"]), _ptr(out["n_act"]), _ptr(out["nnb"])
    return d


# ----------------------------------------------------------------------------
# Calls
# ----------------------------------------------------------------------------
def build_tree(ctx: Context, ds: DeviceState, leaf_size=16, max_depth=21, reorder=False, stream=None):
    perm = torch.empty(max(ds.n, 1), dtype=torch.int32, device=ds.x.device)
    st = ds.struct()
    ctx.check(ctx._lib.sph_build_tree(ctx.h, C.byref(st), int(leaf_size), int(max_depth), int(reorder),
                                      _ptr(perm), _stream(stream)), "sph_build_tree")
    return perm[: ds.n]


def tree_nodes(ctx: Context, cap: int, stream=None):
    dev = "cuda"
    lev = torch.zeros(cap, dtype=torch.int32, device=dev)
    cell = torch.zeros((cap, 3), dtype=torch.int64, device=dev)
    cnt = torch.zeros(cap, dtype=torch.int64, device=dev)
    mass = torch.zeros(cap, dtype=torch.float64, device=dev)
    com = torch.zeros((cap, 3), dtype=torch.float64, device=dev)
    nn = C.c_int64(0)
    ctx.check(ctx._lib.sph_tree_nodes(ctx.h, int(cap), _ptr(lev), _ptr(cell), _ptr(cnt), _ptr(mass), _ptr(com),
                                      C.byref(nn), _stream(stream)), "sph_tree_nodes")
    k = nn.value
    return {"level": lev[:k], "cell": cell[:k], "count": cnt[:k], "mass": mass[:k], "com": com[:k]}


def neighbours(ctx: Context, ds: DeviceState, leaf_size=16, max_depth=21, capacity=None, stream=None):
    cap = capacity if capacity is not None else ds.n * ctx.max_neighbours
    off = torch.zeros(ds.n + 1, dtype=torch.int64, device=ds.x.device)
    idx = torch.zeros(max(cap, 1), dtype=torch.int32, device=ds.x.device)
    st = ds.struct()
    ctx.check(ctx._lib.sph_neighbours(ctx.h, C.byref(st), int(leaf_size), int(max_depth), _ptr(off), _ptr(idx),
                                      int(cap), _stream(stream)), "sph_neighbours")
    return off, idx[: int(off[-1].item())]


def adapt_h(ctx: Context, ds: DeviceState, n_des, tol=0, max_iter=10, leaf_size=16, max_depth=21, stream=None):
    """Variable smoothing length iteration (Sect. 4.2) on ds.h in place.
    Returns (counts of the last pass, number of updates)."""
    cnt = torch.zeros(max(ds.n, 1), dtype=torch.int32, device=ds.x.device)
    upd = C.c_int32(0)
    st = ds.struct()
    ctx.check(ctx._lib.sph_adapt_h(ctx.h, C.byref(st), int(leaf_size), int(max_depth), float(n_des), int(tol),
                                   int(max_iter), _ptr(cnt), C.byref(upd), _stream(stream)), "sph_adapt_h")
    return cnt[: ds.n], upd.value


def flaws(ctx: Context, ds: DeviceState, materials, weibull_k=None, weibull_m=None, seed=0, stream=None):
    """Weibull activation thresholds (Sect. 3.2) of the brittle particles of
    ds.  weibull_k, weibull_m default to the materials' own.  Returns
    (flaw_off int64[n+1] by id, flaw_eps float32) as device tensors; assign
    them to ds.flaw_off / ds.flaw_eps to use them in the damage model."""
    mats, nmat = materials_array(materials), len(materials)
    wk = np.ascontiguousarray([m.weibull_k for m in materials] if weibull_k is None else weibull_k, np.float64)
    wm = np.ascontiguousarray([m.weibull_m for m in materials] if weibull_m is None else weibull_m, np.float64)
    off = torch.zeros(ds.n + 1, dtype=torch.int64, device=ds.x.device)
    tot = C.c_int64(0)
    st = ds.struct()
    seed = int(seed) & (2 ** 64 - 1)
    args = (ctx.h, C.byref(st), mats, nmat, wk.ctypes.data_as(_vp), wm.ctypes.data_as(_vp), seed)
    # a group of N particles takes about N (ln N + 0.58) flaws: size for more,
    # and repeat with the exact total in the (rare) case it does not fit
    cap = int(ds.n * (math.log(max(ds.n, 2)) + 8.0)) + 1024
    eps = torch.empty(cap, dtype=torch.float32, device=ds.x.device)
    r = ctx._lib.sph_flaws(*args, _ptr(off), _ptr(eps), cap, C.byref(tot), _stream(stream))
    if r == SPH_ERR_CAPACITY and tot.value > cap:
        eps = torch.empty(tot.value, dtype=torch.float32, device=ds.x.device)
        r = ctx._lib.sph_flaws(*args, _ptr(off), _ptr(eps), int(tot.value), C.byref(tot), _stream(stream))
    ctx.check(r, "sph_flaws")
    return off, eps[: tot.value]


def fill_flaws(ctx: Context, ps: wl.ParticleSet, stream=None) -> wl.ParticleSet:
    """Draws the Weibull flaws of ps (Sect. 3.2) on the device from
    ps.flaw_seed with the materials' k and m (sph_flaws), into ps.flaw_off and
    ps.flaw_eps (host arrays, indexed by id); returns ps.  No-op when ps has
    its flaws or needs none."""
    from dataclasses import replace
    if ps.flaw_off is not None or getattr(ps, "flaw_seed", None) is None:
        return ps
    ds = DeviceState(replace(ps, flaw_seed=None))
    off, eps = flaws(ctx, ds, ps.materials, seed=ps.flaw_seed, stream=stream)
    ps.flaw_off, ps.flaw_eps = off.cpu().numpy(), eps.cpu().numpy()
    return ps


def fragments(ctx: Context, ds: DeviceState, h0=None, link=1.01, d_remove=1.0, min_size=3, leaf_size=16,
              max_depth=21, stream=None):
    """Friends-of-friends fragments (Sect. 4).  Returns (label int32[n],
    count int32[nf], mass float64[nf]) as device tensors."""
    dev = ds.x.device
    label = torch.empty(max(ds.n, 1), dtype=torch.int32, device=dev)
    cap = max(ds.n, 1)
    cnt = torch.empty(cap, dtype=torch.int32, device=dev)
    mass = torch.empty(cap, dtype=torch.float64, device=dev)
    nf = C.c_int64(0)
    st = ds.struct()
    ctx.check(ctx._lib.sph_fragments(ctx.h, C.byref(st), _ptr(h0), float(link), float(d_remove), int(min_size),
                                     int(leaf_size), int(max_depth), _ptr(label), _ptr(cnt), _ptr(mass), int(cap),
                                     C.byref(nf), _stream(stream)), "sph_fragments")
    return label[: ds.n], cnt[: nf.value], mass[: nf.value]


def neighbours_static(ds: DeviceState, leaf_size=16, max_depth=21, max_neighbours=128, capacity=None,
                      stream=None):
    """Partner lists as ``neighbours`` gives them, through the entry point that
    allocates no device memory (its scratch is a fixed array in the library).
    The output tensors here are allocated by the caller (this function)."""
    L = lib()
    cap = capacity if capacity is not None else ds.n * max_neighbours
    off = torch.zeros(ds.n + 1, dtype=torch.int64, device=ds.x.device)
    idx = torch.zeros(max(cap, 1), dtype=torch.int32, device=ds.x.device)
    st = ds.struct()
    msg = C.create_string_buffer(512)
    r = L.sph_neighbours_static(C.byref(st), int(leaf_size), int(max_depth), int(max_neighbours), _ptr(off),
                                _ptr(idx), int(cap), msg, len(msg), _stream(stream))
    if r != SPH_OK:
        raise SphError(r, "sph_neighbours_static: %s" % msg.value.decode())
    return off, idx[: int(off[-1].item())]


def rhs(ctx: Context, ds: DeviceState, materials, params: wl.Params, out=None, check=True, stream=None):
    out = out if out is not None else alloc_derivs(ds)
    st = ds.struct()
    P = params_struct(params, check)
    d = derivs_struct(out)
    M = materials_array(materials)
    ctx.check(ctx._lib.sph_rhs(ctx.h, C.byref(st), M, len(materials), C.byref(P), C.byref(d), _stream(stream)),
              "sph_rhs")
    return out


def gravity(ctx: Context, ds: DeviceState, params: wl.Params, check=True, stream=None):
    a = torch.zeros((3, max(ds.n, 1)), dtype=torch.float64, device=ds.x.device)
    st = ds.struct()
    P = params_struct(params, check)
    ctx.check(ctx._lib.sph_gravity(ctx.h, C.byref(st), C.byref(P), _ptr(a[0]), _ptr(a[1]), _ptr(a[2]),
                                   _stream(stream)), "sph_gravity")
    return a[: ds.dim, : ds.n]


def step(ctx: Context, ds: DeviceState, materials, params: wl.Params, nsteps: int, check=True, stream=None,
         dt_out=None, cont=False):
    """nsteps predictor-corrector steps (Sect. 3.4.1) in place.  cont: continue
    the tree window the previous step call on ctx left (params.tree_reuse > 0;
    the state must be the one that call returned)."""
    st = ds.struct()
    P = params_struct(params, check, cont)
    M = materials_array(materials)
    dt = dt_out if dt_out is not None else torch.zeros(max(ds.ninst, 1), dtype=torch.float64, device=ds.x.device)
    ctx.check(ctx._lib.sph_step(ctx.h, C.byref(st), M, len(materials), C.byref(P), _ptr(dt), int(nsteps),
                                _stream(stream)), "sph_step")
    return dt


def step_rk3(ctx: Context, ds: DeviceState, materials, params: wl.Params, eps_des: float, nsteps: int, dt=None,
             t=None, check=True, stream=None):
    """nsteps embedded Runge-Kutta attempts (Sect. 3.4.2).  dt, t: per-instance
    device tensors, updated in place (None: new ones; dt <= 0 starts from the
    predictor-corrector limit).  Returns (dt, t, error log, accepted log), the
    logs of shape (nsteps, ninst)."""
    ninst = max(ds.ninst, 1)
    dev = ds.x.device
    dt = dt if dt is not None else torch.zeros(ninst, dtype=torch.float64, device=dev)
    t = t if t is not None else torch.zeros(ninst, dtype=torch.float64, device=dev)
    err = torch.zeros((max(nsteps, 1), ninst), dtype=torch.float64, device=dev)
    acc = torch.zeros((max(nsteps, 1), ninst), dtype=torch.int32, device=dev)
    st = ds.struct()
    P = params_struct(params, check)
    M = materials_array(materials)
    ctx.check(ctx._lib.sph_step_rk3(ctx.h, C.byref(st), M, len(materials), C.byref(P), float(eps_des), _ptr(dt),
                                    _ptr(t), int(nsteps), _ptr(err), _ptr(acc), _stream(stream)), "sph_step_rk3")
    return dt, t, err[:nsteps], acc[:nsteps]


def launch_count() -> int:
    return int(lib().sph_launch_count())


def rhs_adjoint(ctx: Context, ds: DeviceState, materials, params: wl.Params, dbar, sbar: DeviceState,
                param_bar=None, check=True, stream=None):
    """Adds the cotangents of x, v, rho, u, S (into sbar) and of the material
    parameters (into param_bar, shape (ninst, nmat, 3): mu, Y0, K) given the
    cotangents dbar of the right-hand side's outputs (dict like alloc_derivs)."""
    st, sb = ds.struct(), sbar.struct()
    P = params_struct(params, check)
    d = derivs_struct(dbar)
    M = materials_array(materials)
    ctx.check(ctx._lib.sph_rhs_adjoint(ctx.h, C.byref(st), M, len(materials), C.byref(P), C.byref(d), C.byref(sb),
                                       _ptr(param_bar), _stream(stream)), "sph_rhs_adjoint")


def pc_update(ctx: Context, base: DeviceState, d, materials, params: wl.Params, dt, frac, out: DeviceState,
              check=True, stream=None):
    sb, so = base.struct(), out.struct()
    P = params_struct(params, check)
    M = materials_array(materials)
    ctx.check(ctx._lib.sph_pc_update(ctx.h, C.byref(sb), C.byref(derivs_struct(d)), M, len(materials), C.byref(P),
                                     _ptr(dt), float(frac), C.byref(so), _stream(stream)), "sph_pc_update")


def pc_update_adjoint(ctx: Context, base: DeviceState, d, materials, params: wl.Params, dt, frac,
                      out_bar: DeviceState, base_bar: DeviceState, d_bar, param_bar=None, check=True, stream=None):
    sb, ob, bb = base.struct(), out_bar.struct(), base_bar.struct()
    P = params_struct(params, check)
    M = materials_array(materials)
    ctx.check(ctx._lib.sph_pc_update_adjoint(ctx.h, C.byref(sb), C.byref(derivs_struct(d)), M, len(materials),
                                             C.byref(P), _ptr(dt), float(frac), C.byref(ob), C.byref(bb),
                                             C.byref(derivs_struct(d_bar)), _ptr(param_bar), _stream(stream)),
              "sph_pc_update_adjoint")


def measure_fma_peak(precision="mixed"):
    _require_cuda()
    v = C.c_double(0)
    st = lib().sph_measure_fma_peak(PRECISION[precision], C.byref(v))
    if st != SPH_OK:
        raise SphError(st, "sph_measure_fma_peak")
    return v.value


class StepGraph:
    """nsteps predictor-corrector steps captured once as a CUDA graph and
    replayed with replay().  The state arrays of ``ds`` are baked into the
    graph (they are updated in place at every replay); the context must not
    be used by other calls while a replay runs."""

    def __init__(self, ctx: Context, ds: DeviceState, materials, params: wl.Params, nsteps: int = 1):
        self.graph = torch.cuda.CUDAGraph()
        self.stream = torch.cuda.Stream()
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            step(ctx, ds, materials, params, 1, check=False)  # warm-up outside the capture
        torch.cuda.current_stream().wait_stream(self.stream)
        torch.cuda.synchronize()
        self.dt = torch.zeros(max(ds.ninst, 1), dtype=torch.float64, device=ds.x.device)
        with torch.cuda.graph(self.graph, stream=self.stream):
            step(ctx, ds, materials, params, nsteps, check=False, dt_out=self.dt)
        self.ctx = ctx

    def replay(self):
        self.graph.replay()
        return self.dt
