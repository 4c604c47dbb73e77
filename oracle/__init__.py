"""FP64 CPU oracle of the solid-body SPH right-hand side (Schaefer et al. 2016).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_1604_03290_gb300``) never does, and the two share no code.  The
arithmetic lives in ``sph_oracle.c`` (plain C, double precision, built with
``-ffp-contract=off``); this module only compiles it and marshals arguments.

Inputs come as :class:`paper_1604_03290_gb300.workloads.ParticleSet` objects,
plain numpy containers produced by the seeded generators (which hold none of
the method's arithmetic).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

EOS = {"linear": 0, "murnaghan": 1, "tillotson": 2, "isothermal": 3}


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source if it is missing or stale."""
    stale = force or not os.path.exists(_LIB) or max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(_LIB)
    if stale:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Material(C.Structure):
    _fields_ = [("eos", C.c_int32), ("strength", C.c_int32), ("damage", C.c_int32), ("pad", C.c_int32),
                ("rho0", C.c_double), ("cs", C.c_double), ("K0", C.c_double), ("n_M", C.c_double),
                ("A_T", C.c_double), ("B_T", C.c_double), ("E0", C.c_double), ("E_iv", C.c_double),
                ("E_cv", C.c_double), ("a_T", C.c_double), ("b_T", C.c_double), ("alpha_T", C.c_double),
                ("beta_T", C.c_double), ("rho_cut", C.c_double), ("mu", C.c_double), ("Y0", C.c_double)]


class Params(C.Structure):
    _fields_ = [("dim", C.c_int32), ("density_sum", C.c_int32), ("consistency", C.c_int32),
                ("gravity", C.c_int32), ("leaf_size", C.c_int32), ("max_depth", C.c_int32),
                ("alpha", C.c_double), ("beta", C.c_double), ("eps_v", C.c_double),
                ("eps_s", C.c_double), ("n_as", C.c_double), ("dmpd", C.c_double), ("xsph", C.c_double),
                ("G", C.c_double), ("theta", C.c_double), ("eps_grav", C.c_double),
                ("c_courant", C.c_double), ("c_accel", C.c_double), ("c_quantity", C.c_double),
                ("u_floor", C.c_double), ("S_floor", C.c_double), ("dmg_floor", C.c_double),
                ("dt_max", C.c_double), ("dt_fixed", C.c_double), ("n_des", C.c_double),
                ("h_tol", C.c_int32), ("h_iter", C.c_int32), ("tree_reuse", C.c_int32), ("pad2", C.c_int32)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lp = C.POINTER(C.c_int64)
_fp = C.POINTER(C.c_float)


class State(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", _dp), ("y", _dp), ("z", _dp), ("vx", _dp), ("vy", _dp), ("vz", _dp),
                ("rho", _dp), ("u", _dp), ("m", _dp), ("h", _dp), ("S", _dp), ("dmg", _dp), ("mat", _ip),
                ("flaw_off", _lp), ("flaw_eps", _fp), ("id", _ip), ("ninst", C.c_int32), ("pad", C.c_int32),
                ("inst_off", _lp)]


class Derivs(C.Structure):
    _fields_ = [("dxdt", _dp), ("dydt", _dp), ("dzdt", _dp), ("dvx", _dp), ("dvy", _dp), ("dvz", _dp),
                ("drho", _dp), ("du", _dp), ("dS", _dp), ("ddmg", _dp), ("p", _dp), ("cs", _dp),
                ("n_act", _ip), ("nnb", _ip), ("mag_drho", _dp), ("mag_dv", _dp), ("mag_du", _dp),
                ("mag_gradv", _dp), ("mag1_drho", _dp), ("mag1_dv", _dp), ("mag1_du", _dp), ("mag1_gradv", _dp),
                ("mag_rho", _dp), ("mag1_rho", _dp), ("gradv", _dp), ("agx", _dp), ("agy", _dp), ("agz", _dp),
                ("eps_t", _dp)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            L.orc_W.restype = C.c_double
            L.orc_W.argtypes = [C.c_double, C.c_double, C.c_int32]
            L.orc_dWdr.restype = C.c_double
            L.orc_dWdr.argtypes = [C.c_double, C.c_double, C.c_int32]
            L.orc_neighbours_brute.restype = C.c_int64
            L.orc_neighbours_grid.restype = C.c_int64
            L.orc_neighbours_one.restype = C.c_int32
            L.orc_adapt_h.restype = C.c_int32
            L.orc_tree_nodes.restype = C.c_int64
            L.orc_gravity_bh.restype = C.c_int32
            L.orc_rhs.restype = C.c_int32
            L.orc_step.restype = C.c_int32
            L.orc_flaws.restype = C.c_int64
            L.orc_fof.restype = C.c_int64
            L.orc_step_rk3.restype = C.c_int32
            L.orc_get_threads.restype = C.c_int32
            L.orc_eos.argtypes = [C.POINTER(Material), C.c_double, C.c_double, _dp, _dp, _dp, _dp]
            L.orc_sym_eig.argtypes = [C.c_int32, _dp, _dp, _dp]
            _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def _p(a, t=_dp):
    if a is None:
        return C.cast(None, t)
    return a.ctypes.data_as(t)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Marshalling of the seeded inputs
# --------------------------------------------------------------------------
def material_struct(m) -> Material:
    s = Material()
    s.eos = EOS[m.eos]
    s.strength = int(m.strength)
    s.damage = int(m.damage)
    for k in ("rho0", "cs", "K0", "n_M", "A_T", "B_T", "E0", "E_iv", "E_cv", "a_T", "b_T", "alpha_T",
              "beta_T", "rho_cut", "mu", "Y0"):
        setattr(s, k, float(getattr(m, k)))
    return s


def params_struct(p) -> Params:
    s = Params()
    for k, _ in Params._fields_:
        if k == "pad2":
            continue
        v = getattr(p, k)
        setattr(s, k, int(v) if k in ("dim", "density_sum", "consistency", "gravity", "leaf_size", "max_depth",
                                     "h_tol", "h_iter", "tree_reuse") else float(v))
    return s


class _StateArrays:
    """Keeps the numpy buffers of a State alive; fields are copies of the set."""

    def __init__(self, ps, copy=True):
        cp = (lambda a: None if a is None else np.array(a, copy=True)) if copy else (lambda a: a)
        self.dim = ps.dim
        self.n = ps.n
        self.x = cp(_f64(ps.x))
        self.v = cp(_f64(ps.v))
        self.rho = cp(_f64(ps.rho))
        self.u = cp(_f64(ps.u))
        self.m = _f64(ps.m)
        self.h = cp(_f64(ps.h))
        self.S = cp(_f64(ps.S))
        self.dmg = cp(_f64(ps.dmg))
        self.mat = np.ascontiguousarray(ps.mat, dtype=np.int32)
        self.flaw_off = None if ps.flaw_off is None else np.ascontiguousarray(ps.flaw_off, dtype=np.int64)
        self.flaw_eps = None if ps.flaw_eps is None else np.ascontiguousarray(ps.flaw_eps, dtype=np.float32)
        self.id = np.ascontiguousarray(ps.id, dtype=np.int32)
        self.inst_off = None if ps.inst_off is None else np.ascontiguousarray(ps.inst_off, dtype=np.int64)
        self.ninst = ps.ninst
        s = State()
        s.n = self.n
        s.x, s.y = _p(self.x[0]), _p(self.x[1])
        s.z = _p(self.x[2]) if self.dim == 3 else _p(None)
        s.vx, s.vy = _p(self.v[0]), _p(self.v[1])
        s.vz = _p(self.v[2]) if self.dim == 3 else _p(None)
        s.rho, s.u, s.m, s.h = _p(self.rho), _p(self.u), _p(self.m), _p(self.h)
        s.S, s.dmg = _p(self.S), _p(self.dmg)
        s.mat = _p(self.mat, _ip)
        s.flaw_off = _p(self.flaw_off, _lp)
        s.flaw_eps = _p(self.flaw_eps, _fp)
        s.id = _p(self.id, _ip)
        s.ninst = self.ninst
        s.inst_off = _p(self.inst_off, _lp)
        self.struct = s

    def as_dict(self):
        return {"x": self.x, "v": self.v, "rho": self.rho, "u": self.u, "S": self.S, "dmg": self.dmg, "h": self.h}


def _derivs(dim, n, ns):
    out = {
        "dxdt": np.zeros((dim, n)), "dv": np.zeros((dim, n)), "drho": np.zeros(n), "du": np.zeros(n),
        "dS": np.zeros((ns, n)), "ddmg": np.zeros(n), "p": np.zeros(n), "cs": np.zeros(n),
        "n_act": np.zeros(n, np.int32), "nnb": np.zeros(n, np.int32), "mag_drho": np.zeros(n),
        "mag_dv": np.zeros(n), "mag_du": np.zeros(n), "mag_gradv": np.zeros(n),
        "gradv": np.zeros((dim * dim, n)), "ag": np.zeros((dim, n)), "mag1_drho": np.zeros(n),
        "mag1_dv": np.zeros(n), "mag1_du": np.zeros(n), "mag1_gradv": np.zeros(n), "mag_rho": np.zeros(n),
        "mag1_rho": np.zeros(n), "eps_t": np.zeros(n),
    }
    d = Derivs()
    d.dxdt, d.dydt = _p(out["dxdt"][0]), _p(out["dxdt"][1])
    d.dzdt = _p(out["dxdt"][2]) if dim == 3 else _p(None)
    d.dvx, d.dvy = _p(out["dv"][0]), _p(out["dv"][1])
    d.dvz = _p(out["dv"][2]) if dim == 3 else _p(None)
    d.drho, d.du, d.dS, d.ddmg = _p(out["drho"]), _p(out["du"]), _p(out["dS"]), _p(out["ddmg"])
    d.p, d.cs = _p(out["p"]), _p(out["cs"])
    d.n_act, d.nnb = _p(out["n_act"], _ip), _p(out["nnb"], _ip)
    d.mag_drho, d.mag_dv, d.mag_du = _p(out["mag_drho"]), _p(out["mag_dv"]), _p(out["mag_du"])
    d.mag_gradv, d.gradv = _p(out["mag_gradv"]), _p(out["gradv"])
    d.mag1_drho, d.mag1_dv, d.mag1_du = _p(out["mag1_drho"]), _p(out["mag1_dv"]), _p(out["mag1_du"])
    d.mag1_gradv, d.mag_rho, d.mag1_rho = _p(out["mag1_gradv"]), _p(out["mag_rho"]), _p(out["mag1_rho"])
    d.agx, d.agy = _p(out["ag"][0]), _p(out["ag"][1])
    d.agz = _p(out["ag"][2]) if dim == 3 else _p(None)
    d.eps_t = _p(out["eps_t"])
    return d, out


def _mats(materials):
    arr = (Material * len(materials))()
    for i, m in enumerate(materials):
        arr[i] = material_struct(m)
    return arr


# --------------------------------------------------------------------------
# Public oracle calls
# --------------------------------------------------------------------------
def W(r, h, dim):
    return lib().orc_W(float(r), float(h), int(dim))


def dWdr(r, h, dim):
    return lib().orc_dWdr(float(r), float(h), int(dim))


def _xyz(x, dim):
    x = _f64(x)
    return x, _p(x[0]), _p(x[1]), (_p(x[2]) if dim == 3 else _p(None))


def neighbours(x, h, dim, method="grid"):
    """CSR (offsets int64[n+1], indices int32) of N(a) = {b != a: r < (h_a+h_b)/2}."""
    x, px, py, pz = _xyz(x, dim)
    h = _f64(h)
    n = x.shape[1]
    off = np.zeros(n + 1, np.int64)
    cap = max(64 * n, 1024)
    fn = lib().orc_neighbours_grid if method == "grid" else lib().orc_neighbours_brute
    while True:
        idx = np.zeros(cap, np.int32)
        tot = fn(C.c_int32(dim), C.c_int64(n), px, py, pz, _p(h), _p(off, _lp), _p(idx, _ip), C.c_int64(cap))
        if tot >= 0:
            return off, idx[:tot].copy()
        cap = int(off[n]) + 1


def neighbours_one(x, h, dim, a, cap=4096):
    x, px, py, pz = _xyz(x, dim)
    h = _f64(h)
    out = np.zeros(cap, np.int32)
    c = lib().orc_neighbours_one(C.c_int32(dim), C.c_int64(x.shape[1]), px, py, pz, _p(h), C.c_int64(a),
                                 _p(out, _ip), C.c_int32(cap))
    assert c <= cap
    return out[:c].copy()


def adapt_h(x, h, dim, n_des, tol=0, max_iter=10, inst_off=None):
    """Variable smoothing length iteration (Sect. 4.2).  Returns (h, counts,
    number of updates); the input h is not modified."""
    x, px, py, pz = _xyz(x, dim)
    n = x.shape[1]
    hh = np.array(h, dtype=np.float64, copy=True)
    cnt = np.zeros(max(n, 1), np.int32)
    io = None if inst_off is None else np.ascontiguousarray(inst_off, dtype=np.int64)
    ninst = 1 if io is None else len(io) - 1
    it = lib().orc_adapt_h(C.c_int32(dim), C.c_int64(n), px, py, pz, _p(hh), _p(io, _lp), C.c_int32(ninst),
                           C.c_double(n_des), C.c_int32(tol), C.c_int32(max_iter), _p(cnt, _ip))
    return hh, cnt[:n], int(it)


def philox4x64(ctr, key):
    """One Philox4x64-10 block: four 64-bit words (Python ints)."""
    c = (C.c_uint64 * 4)(*[int(v) & (2 ** 64 - 1) for v in ctr])
    k = (C.c_uint64 * 2)(*[int(v) & (2 ** 64 - 1) for v in key])
    out = (C.c_uint64 * 4)()
    lib().orc_philox4x64(c, k, out)
    return [int(v) for v in out]


def flaws(ps, weibull_k=None, weibull_m=None, seed=0):
    """Weibull activation thresholds (Sect. 3.2) of the particle set's brittle
    groups (instance x material).  weibull_k, weibull_m default to the
    materials' own.  Returns (flaw_off int64[n+1] by id, flaw_eps float32)."""
    n = ps.n
    nmat = len(ps.materials)
    wk = np.array([m.weibull_k for m in ps.materials] if weibull_k is None else weibull_k, np.float64)
    wm = np.array([m.weibull_m for m in ps.materials] if weibull_m is None else weibull_m, np.float64)
    mats = _mats(ps.materials)
    ids = np.ascontiguousarray(ps.id, np.int32)
    mat = np.ascontiguousarray(ps.mat, np.int32)
    m = _f64(ps.m)
    io = None if ps.inst_off is None else np.ascontiguousarray(ps.inst_off, np.int64)
    ninst = 1 if io is None else len(io) - 1
    off = np.zeros(n + 1, np.int64)
    cap = int(n * (np.log(max(n, 2)) + 12)) + 64
    while True:
        eps = np.zeros(max(cap, 1), np.float32)
        tot = lib().orc_flaws(C.c_int64(n), _p(ids, _ip), _p(mat, _ip), _p(m), _p(io, _lp), C.c_int32(ninst),
                              mats, C.c_int32(nmat), _p(wk), _p(wm), C.c_uint64(seed), _p(off, _lp),
                              _p(eps, _fp), C.c_int64(cap))
        if tot < 0:
            raise ValueError("ids are not a permutation of 0..n-1")
        if tot <= cap:
            return off, eps[:tot]
        cap = tot


def fof(x, h0, m, dim, b=1.01, d_remove=1.0, min_size=3, dmg=None, inst_off=None):
    """Friends-of-friends fragments (Sect. 4).  Returns (label int32[n],
    count int32[nf], mass float64[nf])."""
    x, px, py, pz = _xyz(x, dim)
    n = x.shape[1]
    h0 = _f64(h0)
    m = _f64(m)
    dm = None if dmg is None else _f64(dmg)
    io = None if inst_off is None else np.ascontiguousarray(inst_off, np.int64)
    ninst = 1 if io is None else len(io) - 1
    label = np.zeros(max(n, 1), np.int32)
    cap = max(n, 1)
    cnt = np.zeros(cap, np.int32)
    mass = np.zeros(cap)
    nf = lib().orc_fof(C.c_int32(dim), C.c_int64(n), px, py, pz, _p(h0), _p(dm), _p(m), _p(io, _lp),
                       C.c_int32(ninst), C.c_double(b), C.c_double(d_remove), C.c_int32(min_size), _p(label, _ip),
                       _p(cnt, _ip), _p(mass), C.c_int64(cap))
    return label[:n], cnt[:nf], mass[:nf]


def cell_coords(x, dim, max_depth=21):
    x, px, py, pz = _xyz(x, dim)
    n = x.shape[1]
    k = np.zeros((n, 3), np.int64)
    lib().orc_cell_coords(C.c_int32(dim), C.c_int64(n), px, py, pz, C.c_int32(max_depth), _p(k, _lp))
    return k


def tree_nodes(x, m, dim, leaf_size, max_depth=21):
    """Pre-order node list: level, cell (n,3), count, mass, com (n,3)."""
    x, px, py, pz = _xyz(x, dim)
    m = _f64(m)
    n = x.shape[1]
    cap = 4 * n + 1024
    while True:
        lev = np.zeros(cap, np.int32)
        cell = np.zeros((cap, 3), np.int64)
        cnt = np.zeros(cap, np.int64)
        mass = np.zeros(cap)
        com = np.zeros((cap, 3))
        nn = lib().orc_tree_nodes(C.c_int32(dim), C.c_int64(n), px, py, pz, _p(m), C.c_int32(leaf_size),
                                  C.c_int32(max_depth), C.c_int64(cap), _p(lev, _ip), _p(cell, _lp),
                                  _p(cnt, _lp), _p(mass), _p(com))
        if nn >= 0:
            return {"level": lev[:nn], "cell": cell[:nn], "count": cnt[:nn], "mass": mass[:nn], "com": com[:nn]}
        cap *= 2


def gravity_direct(x, m, h, dim, G, eps_grav):
    x, px, py, pz = _xyz(x, dim)
    n = x.shape[1]
    a = np.zeros((3, n))
    lib().orc_gravity_direct(C.c_int32(dim), C.c_int64(n), px, py, pz, _p(_f64(m)), _p(_f64(h)),
                             C.c_double(G), C.c_double(eps_grav), _p(a[0]), _p(a[1]), _p(a[2]))
    return a[:dim]


def gravity_bh_reuse(xb, x, m, h, dim, G, theta, eps_grav, leaf_size, max_depth=21):
    """Barnes-Hut accelerations at x with the tree and pseudo-particles of xb."""
    xb, pxb, pyb, pzb = _xyz(xb, dim)
    x, px, py, pz = _xyz(x, dim)
    n = x.shape[1]
    out = np.zeros((3, n))
    lib().orc_gravity_bh_reuse(C.c_int32(dim), C.c_int64(n), pxb, pyb, pzb, px, py, pz, _p(_f64(m)), _p(_f64(h)),
                               C.c_double(G), C.c_double(theta), C.c_double(eps_grav), C.c_int32(leaf_size),
                               C.c_int32(max_depth), None, C.c_int64(0), _p(out[0]), _p(out[1]), _p(out[2]))
    return out[:dim]


def gravity_bh(x, m, h, dim, G, theta, eps_grav, leaf_size, max_depth=21, sample=None):
    x, px, py, pz = _xyz(x, dim)
    n = x.shape[1]
    smp = None if sample is None else np.ascontiguousarray(sample, dtype=np.int64)
    cnt = n if smp is None else len(smp)
    a = np.zeros((3, max(cnt, 1)))
    lib().orc_gravity_bh(C.c_int32(dim), C.c_int64(n), px, py, pz, _p(_f64(m)), _p(_f64(h)), C.c_double(G),
                         C.c_double(theta), C.c_double(eps_grav), C.c_int32(leaf_size), C.c_int32(max_depth),
                         _p(smp, _lp), C.c_int64(cnt), _p(a[0]), _p(a[1]), _p(a[2]))
    return a[:dim, :cnt]


def eos(material, rho, u):
    """(p, dp/drho, dp/du, c_s) of one state."""
    m = material_struct(material)
    out = [C.c_double() for _ in range(4)]
    lib().orc_eos(C.byref(m), float(rho), float(u), *[C.byref(o) for o in out])
    return tuple(o.value for o in out)


def sym_eig(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    dim = A.shape[0]
    w = np.zeros(dim)
    V = np.zeros((dim, dim))
    lib().orc_sym_eig(C.c_int32(dim), _p(A), _p(w), _p(V))
    return w, V


def ensure_flaws(ps):
    """Draws the particle set's Weibull flaws with orc_flaws (Sect. 3.2) from
    its flaw_seed when they are still missing, in place; returns ps."""
    if ps.flaw_off is None and getattr(ps, "flaw_seed", None) is not None:
        ps.flaw_off, ps.flaw_eps = flaws(ps, seed=ps.flaw_seed)
    return ps


def rhs(ps, materials, params):
    """One right-hand side.  Returns a dict of derivatives and diagnostics;
    ``rho`` holds the (possibly recomputed) density."""
    ensure_flaws(ps)
    st = _StateArrays(ps)
    ns = 6 if ps.dim == 3 else 3
    d, out = _derivs(ps.dim, ps.n, ns)
    P = params_struct(params)
    M = _mats(materials)
    rc = lib().orc_rhs(C.byref(st.struct), M, C.c_int32(len(materials)), C.byref(P), C.byref(d))
    if rc != 0:
        raise RuntimeError("oracle rhs failed: %d" % rc)
    out["rho"] = st.rho
    return out


def timestep(ps, materials, params, derivs):
    ensure_flaws(ps)
    st = _StateArrays(ps)
    d = Derivs()
    dim = ps.dim
    keep = {k: np.ascontiguousarray(v) for k, v in derivs.items() if isinstance(v, np.ndarray)}
    d.dvx, d.dvy = _p(keep["dv"][0]), _p(keep["dv"][1])
    d.dvz = _p(keep["dv"][2]) if dim == 3 else _p(None)
    d.drho, d.du, d.cs = _p(keep["drho"]), _p(keep["du"]), _p(keep["cs"])
    d.dS = _p(keep["dS"]) if ps.S is not None else _p(None)
    d.ddmg = _p(keep["ddmg"]) if ps.dmg is not None else _p(None)
    dt = np.zeros(max(ps.ninst, 1))
    lib().orc_timestep(C.byref(st.struct), _mats(materials), C.c_int32(len(materials)),
                       C.byref(params_struct(params)), C.byref(d), _p(dt))
    return dt


def step_rk3(ps, materials, params, eps_des, nsteps, dt=None, t=None):
    """nsteps embedded Runge-Kutta attempts (Sect. 3.4.2) on a copy.  dt, t: per
    instance (None: dt from the predictor-corrector limit, t = 0).  Returns
    (state dict, dt, t, error log [nsteps, ninst], accepted log [nsteps, ninst])."""
    ensure_flaws(ps)
    st = _StateArrays(ps)
    ninst = max(ps.ninst, 1)
    dtv = np.zeros(ninst) if dt is None else np.array(dt, dtype=np.float64, copy=True)
    tv = np.zeros(ninst) if t is None else np.array(t, dtype=np.float64, copy=True)
    err = np.zeros((max(nsteps, 1), ninst))
    acc = np.zeros((max(nsteps, 1), ninst), np.int32)
    rc = lib().orc_step_rk3(C.byref(st.struct), _mats(materials), C.c_int32(len(materials)),
                            C.byref(params_struct(params)), C.c_double(eps_des), C.c_int32(nsteps), _p(dtv),
                            _p(tv), _p(err), _p(acc, _ip))
    if rc != 0:
        raise RuntimeError("oracle rk3 step failed: %d" % rc)
    return st.as_dict(), dtv, tv, err[:nsteps], acc[:nsteps]


def step(ps, materials, params, nsteps):
    """Run nsteps predictor-corrector steps on a copy; returns (state dict, dt log [nsteps, ninst])."""
    ensure_flaws(ps)
    st = _StateArrays(ps)
    ninst = max(ps.ninst, 1)
    dt = np.zeros(ninst)
    log = np.zeros((max(nsteps, 1), ninst))
    rc = lib().orc_step(C.byref(st.struct), _mats(materials), C.c_int32(len(materials)),
                        C.byref(params_struct(params)), C.c_int32(nsteps), _p(dt), _p(log))
    if rc != 0:
        raise RuntimeError("oracle step failed: %d" % rc)
    return st.as_dict(), log[:nsteps]
