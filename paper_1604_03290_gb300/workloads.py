"""Seeded synthetic particle sets shaped like the paper's test problems.

This module only *creates inputs*: lattices, jitter, masses, velocities,
material and run parameters.  It holds none of the method's arithmetic.  The
Weibull flaws the damage model needs (Sect. 3.2) are not drawn here: a damage
workload carries the seed of its flaws (``flaw_seed``), and the flaw
generator of the library (sph_flaws) or of the oracle (orc_flaws), pinned
against each other, draws them from it.  Both the CUDA path and the CPU
oracle are fed from this module, so neither one's input depends on the
other.

Units are SI except for the 2D ring problem, which uses the paper's code units
(length cm, density rho0, velocity c_s; Sect. 4.1).

Workloads (all seeded with ``numpy.random.default_rng(seed)``):

* :func:`rings_2d`        two elastic rubber rings (Sect. 4.1), ~4.4k particles
* :func:`al_impact`       aluminium sphere into aluminium cube (Sect. 4.3)
* :func:`measurement_1m`  the same physics at 100^3 cube particles with a
                          perturbed state that exercises every branch
* :func:`cloud_collapse`  isothermal rotating cloud with self-gravity (Sect. 4.2)
* :func:`ceres_pair`      two basalt bodies with damage and gravity (Sect. 5)
* :func:`batched_impacts` many independent basalt impacts of uneven size
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

G_SI = 6.674e-11
M_SUN = 1.989e30
K_BOLTZMANN = 1.380649e-23
M_HYDROGEN = 1.6735575e-27


@dataclass
class Material:
    """Material parameters of Sect. 2.5-2.7.  ``K0`` is the bulk modulus that
    enters Young's modulus and the crack speed (for Tillotson materials the
    paper sets A_T and B_T equal to it, Table 1)."""
    name: str = ""
    eos: str = "linear"          # linear | murnaghan | tillotson | isothermal
    rho0: float = 1.0
    cs: float = 0.0
    K0: float = 0.0
    n_M: float = 1.0
    A_T: float = 0.0
    B_T: float = 0.0
    E0: float = 1.0
    E_iv: float = 0.0
    E_cv: float = 1.0
    a_T: float = 0.0
    b_T: float = 0.0
    alpha_T: float = 0.0
    beta_T: float = 0.0
    rho_cut: float = 0.0
    mu: float = 0.0
    Y0: float = 0.0              # <= 0: no yield limit
    strength: bool = False
    damage: bool = False
    weibull_k: float = 0.0
    weibull_m: float = 0.0


@dataclass
class Params:
    """Run parameters (artificial viscosity and stress, XSPH, gravity, time
    step factors, precision).  Defaults are the paper's where it gives one."""
    dim: int = 3
    alpha: float = 1.0
    beta: float = 2.0
    eps_v: float = 0.01
    eps_s: float = 0.0
    n_as: float = 4.0
    dmpd: float = 1.0
    xsph: float = 0.0
    density_sum: bool = False
    consistency: bool = True
    gravity: bool = False
    G: float = G_SI
    theta: float = 0.5
    eps_grav: float = 0.5
    leaf_size: int = 16
    max_depth: int = 21
    c_courant: float = 0.7
    c_accel: float = 0.2
    c_quantity: float = 0.7
    u_floor: float = 1.0
    S_floor: float = 1.0
    dmg_floor: float = 1e-2
    dt_max: float = 1e30
    dt_fixed: float = 0.0
    n_des: float = 0.0           # > 0: variable h at each step start (Sect. 4.2)
    h_tol: int = 0
    h_iter: int = 8
    tree_reuse: int = 0          # > 0: one tree serves this many steps (decoupled self-gravity)
    precision: str = "fp64"      # fp64 | mixed


@dataclass
class ParticleSet:
    dim: int
    x: np.ndarray                # (dim, n) float64
    v: np.ndarray                # (dim, n)
    rho: np.ndarray
    u: np.ndarray
    m: np.ndarray
    h: np.ndarray
    mat: np.ndarray              # int32
    id: np.ndarray               # int32, original index (flaws are indexed by it)
    S: Optional[np.ndarray] = None      # (3 or 6, n) component-major
    dmg: Optional[np.ndarray] = None    # d^(1/3)
    flaw_off: Optional[np.ndarray] = None   # int64 (n+1), indexed by id
    flaw_eps: Optional[np.ndarray] = None   # float32, ascending per particle
    flaw_seed: Optional[int] = None         # seed of the flaws still to draw (flaw_off is None until then)
    inst_off: Optional[np.ndarray] = None   # int64 (ninst+1)
    materials: List[Material] = field(default_factory=list)
    params: Params = field(default_factory=Params)
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.x.shape[1])

    @property
    def ninst(self) -> int:
        return 1 if self.inst_off is None else int(len(self.inst_off) - 1)

    @property
    def nsym(self) -> int:
        return 6 if self.dim == 3 else 3

    def copy(self) -> "ParticleSet":
        c = lambda a: None if a is None else a.copy()
        return replace(self, x=c(self.x), v=c(self.v), rho=c(self.rho), u=c(self.u), m=c(self.m), h=c(self.h),
                       mat=c(self.mat), id=c(self.id), S=c(self.S), dmg=c(self.dmg))

    def subset_order(self, order: np.ndarray) -> "ParticleSet":
        """The same particles in another order (flaws stay indexed by id)."""
        t = lambda a: None if a is None else a[..., order].copy()
        return replace(self, x=t(self.x), v=t(self.v), rho=t(self.rho), u=t(self.u), m=t(self.m), h=t(self.h),
                       mat=t(self.mat), id=t(self.id), S=t(self.S), dmg=t(self.dmg))


# --------------------------------------------------------------------------
# Materials (values as printed in the paper)
# --------------------------------------------------------------------------
def rubber() -> Material:
    """Rubber rings of Sect. 4.1 in code units: rho0 = 1, c_s = 1, mu = 0.22."""
    return Material(name="rubber", eos="linear", rho0=1.0, cs=1.0, K0=1.0, mu=0.22, Y0=0.0, strength=True)


def aluminium_6061() -> Material:
    """Al 6061 of Sect. 4.3: Tillotson parameters, mu, K0, Y0."""
    return Material(name="Al6061", eos="tillotson", rho0=2.7e3, K0=75.27e9, A_T=75.2e9, B_T=65e9, E0=5e6,
                    E_iv=3e6, E_cv=13.9e6, a_T=0.5, b_T=1.63, alpha_T=5.0, beta_T=5.0, mu=26e9, Y0=1e8,
                    strength=True)


def basalt() -> Material:
    """Basalt of Table 1 (Tillotson, mu, Y0) and Table 2 (Weibull k, m)."""
    return Material(name="basalt", eos="tillotson", rho0=2700.0, K0=26.7e9, A_T=26.7e9, B_T=26.7e9, E0=487e6,
                    E_iv=4.72e6, E_cv=18.2e6, a_T=0.5, b_T=1.5, alpha_T=5.0, beta_T=5.0, mu=22.7e9, Y0=3.5e9,
                    strength=True, damage=True, weibull_k=1e61, weibull_m=16.0)


def ice() -> Material:
    """Water ice of Tables 1 and 2."""
    return Material(name="ice", eos="tillotson", rho0=917.0, K0=9.47e9, A_T=9.47e9, B_T=9.47e9, E0=10e6,
                    E_iv=0.773e6, E_cv=3.04e6, a_T=0.3, b_T=0.1, alpha_T=10.0, beta_T=5.0, mu=2.8e9, Y0=1e9,
                    strength=True, damage=True, weibull_k=1e46, weibull_m=9.1)


def molecular_hydrogen_10K() -> Material:
    """Isothermal ideal gas of pure H2 at T = 10 K (Sect. 4.2)."""
    cs = math.sqrt(K_BOLTZMANN * 10.0 / (2.0 * M_HYDROGEN))
    return Material(name="H2-10K", eos="isothermal", rho0=1.44e-14, cs=cs)


# --------------------------------------------------------------------------
# Helpers
# --------------------------------------------------------------------------
def _lattice_box(nx, ny, nz, dx, origin=(0.0, 0.0, 0.0)):
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    pts = np.stack([i.ravel(), j.ravel(), k.ravel()]).astype(np.float64) * dx
    pts += (np.asarray(origin, dtype=np.float64) + 0.5 * dx)[:, None]
    return pts


def _lattice_ball(radius, dx, center=(0.0, 0.0, 0.0)):
    m = int(math.ceil(radius / dx)) + 1
    r = np.arange(-m, m + 1, dtype=np.float64) * dx
    X, Y, Z = np.meshgrid(r, r, r, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
    keep = (pts ** 2).sum(0) <= radius * radius
    return pts[:, keep] + np.asarray(center, dtype=np.float64)[:, None]


def _finish(dim, x, v, m, h, rho, u, mat, materials, params, with_S=True, with_dmg=False, name="",
            inst_off=None):
    n = x.shape[1]
    ns = 6 if dim == 3 else 3
    return ParticleSet(dim=dim, x=np.ascontiguousarray(x, np.float64), v=np.ascontiguousarray(v, np.float64),
                       rho=np.ascontiguousarray(rho, np.float64), u=np.ascontiguousarray(u, np.float64),
                       m=np.ascontiguousarray(m, np.float64), h=np.ascontiguousarray(h, np.float64),
                       mat=np.ascontiguousarray(mat, np.int32), id=np.arange(n, dtype=np.int32),
                       S=np.zeros((ns, n)) if with_S else None, dmg=np.zeros(n) if with_dmg else None,
                       inst_off=inst_off, materials=materials, params=params, name=name)


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------
def rings_2d(seed=1, dx=0.1, h=0.25, r_in=3.0, r_out=4.0, speed=0.059, jitter=1e-3,
             artificial_stress=False) -> ParticleSet:
    """Two rubber rings (Sect. 4.1): annuli r in [3, 4] cm on square lattices
    of spacing dx, centres at x = -/+(r_out + dx), moving at +/-0.059 c_s.
    Config parity run: alpha = 1, beta = 2, fixed dt = 0.3 h / c_s.  With
    ``artificial_stress`` the paper's bounce run: eps_s = 0.2, n = 4,
    XSPH 0.5."""
    rng = np.random.default_rng(seed)
    m_ = int(math.ceil(r_out / dx)) + 1
    g = np.arange(-m_, m_ + 1, dtype=np.float64) * dx
    X, Y = np.meshgrid(g, g, indexing="ij")
    rr = np.sqrt(X ** 2 + Y ** 2)
    keep = (rr >= r_in) & (rr <= r_out)
    ring = np.stack([X[keep], Y[keep]])
    c = r_out + dx
    left = ring + np.array([[-c], [0.0]])
    right = ring + np.array([[c], [0.0]])
    x = np.concatenate([left, right], axis=1)
    x += rng.uniform(-jitter, jitter, size=x.shape)
    n = x.shape[1]
    nl = left.shape[1]
    v = np.zeros((2, n))
    v[0, :nl] = speed
    v[0, nl:] = -speed
    mat = rubber()
    params = Params(dim=2, alpha=1.0, beta=2.0, dmpd=dx, dt_fixed=0.3 * h / mat.cs, u_floor=1e-3, S_floor=1e-3)
    if artificial_stress:
        params = replace(params, eps_s=0.2, n_as=4.0, xsph=0.5)
    return _finish(2, x, v, np.full(n, mat.rho0 * dx * dx), np.full(n, h), np.full(n, mat.rho0), np.zeros(n),
                   np.zeros(n, np.int32), [mat], params, name="rings_2d")


def al_impact(seed=2, n_side=64, side=0.1, sphere_d=0.01, speed=7000.0, mu=27e9, Y0=0.3e9, jitter=0.01,
              h_factor=2.4) -> ParticleSet:
    """Aluminium sphere into aluminium cube (Sect. 4.3 geometry; mu and Y0 as
    given for this workload).  Cube: n_side^3 lattice over `side`; sphere of
    diameter `sphere_d` on a lattice of half the cube spacing, one cube
    spacing above the top face, moving at -speed along z.  Support radius
    h = h_factor * spacing (2.4: Monaghan's 1.2 spacing as a support radius)."""
    rng = np.random.default_rng(seed)
    dx = side / n_side
    cube = _lattice_box(n_side, n_side, n_side, dx, origin=(-side / 2, -side / 2, -side))
    dxp = dx / 2.0
    rs = sphere_d / 2.0
    ball = _lattice_ball(rs, dxp, center=(0.0, 0.0, dx + rs))
    cube += rng.uniform(-jitter, jitter, size=cube.shape) * dx
    ball += rng.uniform(-jitter, jitter, size=ball.shape) * dxp
    x = np.concatenate([cube, ball], axis=1)
    nc, nb = cube.shape[1], ball.shape[1]
    n = nc + nb
    v = np.zeros((3, n))
    v[2, nc:] = -speed
    mat = replace(aluminium_6061(), mu=mu, Y0=Y0)
    h = np.concatenate([np.full(nc, h_factor * dx), np.full(nb, h_factor * dxp)])
    m = np.concatenate([np.full(nc, mat.rho0 * dx ** 3), np.full(nb, mat.rho0 * dxp ** 3)])
    params = Params(dim=3, alpha=0.5, beta=0.0, dmpd=dx, u_floor=1e3, S_floor=1e5)
    return _finish(3, x, v, m, h, np.full(n, mat.rho0), np.zeros(n), np.zeros(n, np.int32), [mat], params,
                   name="al_impact_%d" % n_side)


def measurement_1m(seed=11, n_side=100, damage=True, weibull_k=5e34, weibull_m=8.5) -> ParticleSet:
    """The aluminium-impact physics at n_side^3 cube particles (Delta x = 0.1
    cm for 100^3) plus the projectile, with a state perturbed so that every
    branch runs: rho = rho0 (1 + N(0, 0.01)), u ~ U[0, 1.5e7] J/kg (all three
    Tillotson regimes), v ~ N(0, 10 m/s), S_ij ~ N(0, 0.3 Y0) (some yield),
    d^(1/3) ~ U[0, 0.5] and Weibull flaws (k, m as for the basalt bodies;
    drawn from flaw_seed = seed + 2000)."""
    ps = al_impact(seed=seed, n_side=n_side)
    rng = np.random.default_rng(seed + 1000)
    n = ps.n
    mat = ps.materials[0]
    ps.rho = mat.rho0 * (1.0 + rng.normal(0.0, 0.01, n))
    ps.u = rng.uniform(0.0, 1.5e7, n)
    ps.v = ps.v + rng.normal(0.0, 10.0, (3, n))
    ps.S = rng.normal(0.0, 0.3 * mat.Y0, (6, n))
    if damage:
        mat = replace(mat, damage=True, weibull_k=weibull_k, weibull_m=weibull_m)
        ps.materials = [mat]
        ps.dmg = rng.uniform(0.0, 0.5, n)
        ps.flaw_seed = seed + 2000
    ps.name = "measurement_%d" % n
    return ps


def cloud_collapse(seed=3, n=2_000_000, beta_rot=0.16, amp=0.1, n_des=50, theta=0.5) -> ParticleSet:
    """Rotating isothermal cloud (Sect. 4.2): M = 1 M_sun, R0 = 3.2e14 m,
    jittered cubic lattice (+/-0.3 spacing) cut to the sphere, m = 2 mass
    modulation 1 + amp cos(2 phi), solid rotation with
    Omega = sqrt(3 G M beta / R^3) (beta = rotational / gravitational energy of
    a uniform sphere), h from n_des neighbours, density by kernel sum,
    Barnes-Hut with softening 0.5 h."""
    rng = np.random.default_rng(seed)
    R, M = 3.2e14, M_SUN
    side = (n * 6.0 / math.pi) ** (1.0 / 3.0)
    dx = 2.0 * R / side
    pts = _lattice_ball(R, dx)
    pts += rng.uniform(-0.3, 0.3, size=pts.shape) * dx
    pts = pts[:, (pts ** 2).sum(0) <= R * R]
    npt = pts.shape[1]
    phi = np.arctan2(pts[1], pts[0])
    w = 1.0 + amp * np.cos(2.0 * phi)
    m = M * w / w.sum()
    omega = math.sqrt(3.0 * G_SI * M * beta_rot / R ** 3)
    v = np.zeros_like(pts)
    v[0] = -omega * pts[1]
    v[1] = omega * pts[0]
    ndens = npt / (4.0 / 3.0 * math.pi * R ** 3)
    h = (3.0 * n_des / (4.0 * math.pi * ndens)) ** (1.0 / 3.0)
    mat = molecular_hydrogen_10K()
    params = Params(dim=3, alpha=1.0, beta=2.0, density_sum=True, consistency=False, gravity=True, theta=theta,
                    eps_grav=0.5, dmpd=dx, u_floor=1.0)
    ps = _finish(3, pts, v, m, np.full(npt, h), np.full(npt, mat.rho0), np.zeros(npt), np.zeros(npt, np.int32),
                 [mat], params, with_S=False, name="cloud_%d" % npt)
    return ps


def ceres_pair(seed=4, n_each=1_000_000, R=470e3, speed=1000.0, angle_deg=45.0, theta=0.6) -> ParticleSet:
    """Two basalt bodies (Sect. 5 scenario, sizes as given for this workload):
    radius R each, cubic lattices with +/-0.1 spacing jitter, relative speed
    `speed` with impact parameter 2R sin(angle), one spacing apart at
    contact; Weibull flaws k = 5e34, m = 8.5 (flaw_seed = seed + 2000);
    Barnes-Hut opening angle 0.6."""
    rng = np.random.default_rng(seed)
    dx = R * (4.0 * math.pi / 3.0 / n_each) ** (1.0 / 3.0)
    body = _lattice_ball(R, dx)
    nb = body.shape[1]
    b = 2.0 * R * math.sin(math.radians(angle_deg))
    sep = math.sqrt(max((2.0 * R + dx) ** 2 - b ** 2, 0.0))
    A = body + rng.uniform(-0.1, 0.1, size=body.shape) * dx
    B = body + rng.uniform(-0.1, 0.1, size=body.shape) * dx + np.array([[sep], [b], [0.0]])
    x = np.concatenate([A, B], axis=1)
    n = x.shape[1]
    v = np.zeros((3, n))
    v[0, :nb] = 0.5 * speed
    v[0, nb:] = -0.5 * speed
    mat = replace(basalt(), weibull_k=5e34, weibull_m=8.5)
    params = Params(dim=3, alpha=1.0, beta=2.0, gravity=True, theta=theta, eps_grav=0.5, dmpd=dx,
                    u_floor=1e3, S_floor=1e5)
    ps = _finish(3, x, v, np.full(n, mat.rho0 * dx ** 3), np.full(n, 2.4 * dx), np.full(n, mat.rho0), np.zeros(n),
                 np.zeros(n, np.int32), [mat], params, with_dmg=True, name="ceres_pair_%d" % n)
    ps.flaw_seed = seed + 2000
    return ps


def batched_impacts(seed=5, ninst=256, nmin=2000, nmax=50000, dx=1e-3, vmin=3000.0, vmax=6000.0,
                    with_flaws=True) -> ParticleSet:
    """Independent basalt impacts of uneven size: target particle counts
    log-uniform in [nmin, nmax] (cube or half-ball lattice), a ball projectile
    of 1/64 the target volume on the same spacing, one spacing above the
    target's top, at normal incidence with speed U[vmin, vmax].  Instances
    are concatenated; ``inst_off`` marks them."""
    rng = np.random.default_rng(seed)
    mat = replace(basalt(), weibull_k=5e34, weibull_m=8.5)
    xs, vs, hs, ms = [], [], [], []
    off = [0]
    for i in range(ninst):
        nt = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        if rng.uniform() < 0.5:
            s = int(round(nt ** (1.0 / 3.0)))
            tgt = _lattice_box(s, s, s, dx, origin=(-s * dx / 2, -s * dx / 2, -s * dx))
        else:
            r = (3.0 * nt / (2.0 * math.pi)) ** (1.0 / 3.0) * dx
            tgt = _lattice_ball(r, dx)
            tgt = tgt[:, tgt[2] < 0.0]
        vol_t = tgt.shape[1] * dx ** 3
        rp = (3.0 * vol_t / 64.0 / (4.0 * math.pi)) ** (1.0 / 3.0)
        ztop = tgt[2].max()
        prj = _lattice_ball(max(rp, dx), dx, center=(0.0, 0.0, ztop + dx + max(rp, dx)))
        x = np.concatenate([tgt, prj], axis=1)
        x += rng.uniform(-0.01, 0.01, size=x.shape) * dx
        v = np.zeros_like(x)
        v[2, tgt.shape[1]:] = -rng.uniform(vmin, vmax)
        xs.append(x)
        vs.append(v)
        off.append(off[-1] + x.shape[1])
    x = np.concatenate(xs, axis=1)
    v = np.concatenate(vs, axis=1)
    n = x.shape[1]
    # the Morton key holds 3 * max_depth cell bits plus ceil(log2(ninst))
    # instance bits in 64
    ibits = max(int(ninst - 1).bit_length(), 0)
    params = Params(dim=3, alpha=1.0, beta=2.0, dmpd=dx, u_floor=1e3, S_floor=1e5,
                    max_depth=min(21, (64 - ibits) // 3))
    ps = _finish(3, x, v, np.full(n, mat.rho0 * dx ** 3), np.full(n, 2.4 * dx), np.full(n, mat.rho0), np.zeros(n),
                 np.zeros(n, np.int32), [mat], params, with_dmg=True, name="batched_%d" % ninst,
                 inst_off=np.asarray(off, np.int64))
    if with_flaws:
        ps.flaw_seed = seed + 2000
    return ps


def fragmented_body(seed=21, n_side=100, ncracks=10, dx=1e-3, jitter=0.05, d_spot=0.05) -> ParticleSet:
    """A basalt cube (n_side^3 jittered lattice, h = 2.4 dx) as an impact
    leaves it: fully damaged slabs of half-width 1.3 dx around `ncracks`
    random planes (wider than the 1.01 h linking length, so they cut the body
    into pieces), a fraction d_spot of scattered fully damaged particles, and
    d ~ U[0, 0.95) elsewhere.  The input of the fragment analysis."""
    rng = np.random.default_rng(seed)
    side = n_side * dx
    x = _lattice_box(n_side, n_side, n_side, dx, origin=(-side / 2, -side / 2, -side / 2))
    x += rng.uniform(-jitter, jitter, size=x.shape) * dx
    n = x.shape[1]
    dmg = rng.uniform(0.0, 0.95, n)
    for _ in range(ncracks):
        nrm = rng.normal(size=3)
        nrm /= np.linalg.norm(nrm)
        p0 = rng.uniform(-0.35, 0.35, 3) * side
        dist = np.abs(nrm @ (x - p0[:, None]))
        dmg[dist < 1.3 * dx] = 1.0
    dmg[rng.uniform(size=n) < d_spot] = 1.0
    mat = replace(basalt(), weibull_k=5e34, weibull_m=8.5)
    params = Params(dim=3, alpha=1.0, beta=2.0, dmpd=dx, u_floor=1e3, S_floor=1e5)
    ps = _finish(3, x, np.zeros((3, n)), np.full(n, mat.rho0 * dx ** 3), np.full(n, 2.4 * dx), np.full(n, mat.rho0),
                 np.zeros(n), np.zeros(n, np.int32), [mat], params, with_dmg=True, name="fragmented_%d" % n)
    ps.dmg = dmg
    return ps


def lattice_block(seed=0, nx=12, ny=12, nz=12, dx=1.0, jitter=0.2, h_factor=2.4, dim=3) -> ParticleSet:
    """A small jittered lattice block (unit density, linear EOS) for tests."""
    rng = np.random.default_rng(seed)
    if dim == 3:
        x = _lattice_box(nx, ny, nz, dx)
    else:
        x = _lattice_box(nx, ny, 1, dx)[:2]
    x += rng.uniform(-jitter, jitter, size=x.shape) * dx
    n = x.shape[1]
    mat = Material(name="unit", eos="linear", rho0=1.0, cs=1.0, K0=1.0, mu=0.5, strength=True)
    params = Params(dim=dim, alpha=1.0, beta=2.0, dmpd=dx, u_floor=1e-3, S_floor=1e-3)
    return _finish(dim, x, np.zeros((dim, n)), np.full(n, dx ** dim), np.full(n, h_factor * dx), np.ones(n),
                   np.zeros(n), np.zeros(n, np.int32), [mat], params, name="lattice_block")
