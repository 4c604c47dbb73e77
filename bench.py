#!/usr/bin/env python
"""Throughput of the SPH predictor-corrector step on GB300.

One step = partner search, both neighbour passes with the constitutive
update, the device-side time step and the predictor update, then partners and
passes again at the predicted state and the corrector update (sph_step).  A
tree (and the state's order along it) serves --tree-reuse consecutive steps
(default 5): the step that builds it walks it for the partners, and every
later evaluation of the window refines those lists, exactly, while the
particles' displacement allows (else it walks).  Workload: aluminium sphere into aluminium cube,
Tillotson EOS, strength, von Mises yield and Grady-Kipp damage, 100^3 cube
particles plus a 1 cm projectile (1,004,189 particles), with a perturbed state
so every branch runs.  Metric: particle-updates per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs its own replica
(the single-body workload does not shard), max time over ranks.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SPH step particle-updates/s (mixed precision, 1M-particle Al impact)"
UNIT = "particle-updates/s"
WORKLOAD = ("al_impact_1M: Al6061 cube 100^3 (dx = 1 mm) + 1 cm sphere (dx/2), Tillotson EOS, mu = 27 GPa, "
            "Y0 = 0.3 GPa, Grady-Kipp damage (k = 5e34, m = 8.5), perturbed state (seed 11), "
            "predictor-corrector sph_step, no gravity")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n-side", type=int, default=100)
    ap.add_argument("--fp64-steps", type=int, default=8)
    ap.add_argument("--cpu-side", type=int, default=100, help="cube side of the CPU-baseline sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-aux", action="store_true", help="skip timing the flaw and fragment steps")
    ap.add_argument("--only-aux", action="store_true", help="time only the flaw, fragment and decoupling legs")
    ap.add_argument("--cloud-n", type=int, default=2_000_000, help="particles of the decoupling leg's cloud")
    ap.add_argument("--tree-reuse", type=int, default=5,
                    help="steps one tree serves (partners refined from the build step's walk); 0: a tree per step")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# nvidia-smi clock sampling during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


# ----------------------------------------------------------------------------
# Byte model of the kernels (algorithmic bytes per particle, mixed mode)
# ----------------------------------------------------------------------------
# Per particle and launch, from one ncu capture of the kernels as built (the
# first right-hand side of the warm-up step, after the state is put in tree
# order, and the refine of its predictor evaluation, of the 514,109-particle
# case of this workload, n_side 80; profiles/ holds the summary): warp
# instructions issued (smsp__inst_executed.sum) and DRAM bytes
# (dram__bytes_read.sum + dram__bytes_write.sum).  Both scale with the
# particle count at this density.  "src" is the first 16 hex digits of the
# SHA-256 of the kernel's source file at capture time: when the file differs
# now, the figures are stale and are not used (the kernel is then reported
# against HBM alone, with traffic null).
NCU_PER_PARTICLE = {
    "partners": {"inst": 862.46, "dram": 356.52, "fp32_pipe": 0.274, "issue": 0.683, "l1": 0.328,
                 "src": ("neighbours.cu", "9347fbb88607e52e")},
    "refine": {"inst": 10.60, "dram": 67.06, "fp32_pipe": 0.095, "issue": 0.228, "l1": 0.290,
               "src": ("neighbours.cu", "9347fbb88607e52e")},
    "passA": {"inst": 315.03, "dram": 499.16, "fp32_pipe": 0.384, "issue": 0.582, "l1": 0.695,
              "src": ("rhs.cu", "34f6a376fba94640")},
    "passB": {"inst": 336.22, "dram": 347.92, "fp32_pipe": 0.416, "issue": 0.567, "l1": 0.889,
              "src": ("rhs.cu", "34f6a376fba94640")},
}


def ncu_figures(phase):
    """The captured per-particle figures of `phase` if its source is unchanged."""
    import hashlib
    c = NCU_PER_PARTICLE.get(phase)
    if not c:
        return None
    fn, sha = c["src"]
    with open(os.path.join(ROOT, "paper_1604_03290_gb300", "csrc", fn), "rb") as f:
        now = hashlib.sha256(f.read()).hexdigest()[:16]
    return c if now == sha else None
ISSUE_SLOTS_PER_SM = 4  # one warp instruction per clock per SM sub-partition


def algorithmic_bytes(phase, K, n_flaw_mean, dim=3):
    """HBM bytes one particle must move in one launch of `phase`, counting each
    array once (partner data reused from cache): K = mean partners."""
    ns = 6 if dim == 3 else 3
    lg = math.log2(max(n_flaw_mean, 1.0)) + 1.0
    if phase == "passA":
        reads = 64 + 8 + 8 + 8 * ns + 8 + 4 + 4 + 16 + 4 * lg + 4 + 4 * K  # packs, rho, u, S, dmg, mat, id, flaws, list
        writes = 8 + 8 * dim + 8 * ns + 8 + 4 + 32  # drho, dx, dS, ddmg, n_act, T pack
        return reads + writes
    if phase == "passB":
        return 64 + 32 + 4 + 4 * K + 8 * dim + 8  # packs, T pack, list; dv, du
    # the shell of the later evaluations: candidates with (1 - 1/64) h_ab <=
    # r_ab < (1 + 1/64) h_ab, about ((1 + 1/64)^D - (1 - 1/64)^D) K of them for
    # uniformly spread neighbours (fewer on the bench lattice)
    shell = ((1.0 + 1.0 / 64.0) ** dim - (1.0 - 1.0 / 64.0) ** dim) * K
    if phase == "partners":
        # positions, perm, slot; list and count; the shell list and its count
        return 32 + 4 + 4 + 4 * K + 4 + 4 * shell + 4
    if phase == "refine":
        # per particle: counts, shell bits and h, own positions, the shell and
        # its members' positions (gathered: 32 B each), the new count; the old
        # list is read and a new one written only where a shell member changed
        # sides (none on the bench workload's lattice)
        return 4 + 4 + 4 + 8 + 32 + 36 * shell + 4
    raise KeyError(phase)


# ----------------------------------------------------------------------------
# Steps on either side of the damage path, timed outside the step: the Weibull
# flaw distribution of the measured configuration (Sect. 3.2) and the
# friends-of-friends fragments of a 1M-particle fragmented body (Sect. 4).
# ----------------------------------------------------------------------------
def oracle_time(fn):
    """Seconds of one oracle call on all host cores (the oracle as it stands)."""
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    oracle.set_threads(cores)
    t0 = time.perf_counter()
    fn(oracle)
    return time.perf_counter() - t0, cores


def adjoint_rollout(sph, wl, stream, nsteps=50, every=10):
    """Gradients of the penetration depth of 256 batched impacts after 50
    fixed steps with respect to each impact speed and to mu, Y0 and K, by the
    checkpointed adjoint (a checkpoint every 10 steps, damage off), mixed
    precision: forward and backward time and the device memory they use."""
    import numpy as np
    import torch
    from dataclasses import replace
    from paper_1604_03290_gb300 import adjoint
    bt = wl.batched_impacts(seed=5, with_flaws=False)
    mat = replace(bt.materials[0], damage=False)
    bt.materials, bt.dmg = [mat], None
    cmax = float(np.sqrt(mat.A_T / mat.rho0))
    dt = 0.25 * float(bt.h.min()) / (cmax + 6000.0)
    prm = replace(bt.params, max_depth=18, alpha=1.0, beta=2.0, dt_fixed=dt, precision="mixed")
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    base = torch.cuda.memory_allocated()
    ctx = sph.Context(3, bt.n, max_instances=bt.ninst, max_neighbours=128, leaf_size=prm.leaf_size)
    proj = torch.as_tensor((bt.v[2] < 0).astype(np.float64), device="cuda")
    inst = torch.as_tensor(np.repeat(np.arange(bt.ninst), np.diff(bt.inst_off)), device="cuda")
    x0 = torch.as_tensor(bt.x, device="cuda")
    m = torch.as_tensor(bt.m, device="cuda")
    # warm-up: one checkpoint segment forward and back (loads the kernels and
    # fills the allocator's pool with the segment's states), not timed
    warm = adjoint.Runner(ctx, bt, prm, dt, every, every=every)
    vw = torch.as_tensor(bt.v, device="cuda").requires_grad_(True)
    tw = adjoint.theta_of(bt.materials).requires_grad_(True)
    xw, _ = adjoint.rollout(warm, bt.materials, x0, vw, tw)
    adjoint.penetration_depth(xw, m, proj, 0.0, inst, bt.ninst).sum().backward()
    del warm, xw, vw, tw
    runner = adjoint.Runner(ctx, bt, prm, dt, nsteps, every=every)
    v0 = torch.as_tensor(bt.v, device="cuda").requires_grad_(True)
    theta = adjoint.theta_of(bt.materials).requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xN, vN = adjoint.rollout(runner, bt.materials, x0, v0, theta)
    J = adjoint.penetration_depth(xN, m, proj, 0.0, inst, bt.ninst)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    J.sum().backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    g_speed = -(v0.grad[2] * proj).cpu().numpy()
    per_inst = np.bincount(inst.cpu().numpy(), weights=g_speed, minlength=bt.ninst)
    out = {"workload": "%d batched basalt impacts (%d particles), %d fixed steps of %.3g s, checkpoint every %d, "
                       "mixed precision, damage off" % (bt.ninst, bt.n, nsteps, dt, every),
           "forward_s": t1 - t0, "backward_s": t2 - t1,
           "particle_steps_per_s": bt.n * nsteps / (t2 - t0),
           "peak_torch_bytes": torch.cuda.max_memory_allocated() - base, "context_bytes": ctx.bytes,
           "dJ_dV0_range": [float(per_inst.min()), float(per_inst.max())],
           "dJ_dtheta": [float(v) for v in theta.grad.numpy()[0]]}
    del runner, ctx
    return out


def aux_rows(sph, wl, ctx, ps, stream, hbm_peak, reps=3, cloud_n=2_000_000, with_oracle=False):
    import numpy as np
    import torch
    from dataclasses import replace

    def timed(fn, ctx=ctx):
        fn()  # warm-up
        ctx.sync_status()
        ctx.profile(True)
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ph = ctx.profile_read()
        ctx.profile(False)
        phases = {k: v[0] / reps for k, v in ph.items() if v[1] > 0}
        return statistics.median(ts), phases, out

    ds = sph.DeviceState(ps)
    ms_f, ph_f, (off, eps) = timed(lambda: sph.flaws(ctx, ds, ps.materials, seed=12345))
    nfl = int(eps.numel())
    flaws = {"workload": "Weibull flaws of the measured configuration (%d particles, k = %g, m = %g, seed 12345)"
                         % (ps.n, ps.materials[0].weibull_k, ps.materials[0].weibull_m),
             "ms": ms_f, "flaws": nfl, "value": nfl / (ms_f * 1e-3), "unit": "flaws/s", "phases_ms": ph_f,
             # output bytes: thresholds (4 B each) and offsets (8 B per particle)
             "hbm_frac_output_bytes": (4 * nfl + 8 * ps.n) / (ms_f * 1e-3) / 1e9 / hbm_peak}
    if with_oracle:
        sec, cores = oracle_time(lambda o: o.flaws(ps, seed=12345))
        flaws["cpu_baseline"] = {"value": nfl / sec, "unit": "flaws/s", "cores": cores, "kind": "oracle",
                                 "sample": "the same call on the host (%.1f s)" % sec}
    del ds, off, eps
    fb = wl.fragmented_body(seed=21)
    dsf = sph.DeviceState(fb)
    # the bench's context when it holds the body (a smaller --n-side: one of its own)
    ctxf = ctx if fb.n <= ctx.max_particles else sph.Context(3, fb.n, max_neighbours=ctx.max_neighbours)
    ms_g, ph_g, (lab, cnt, mass) = timed(lambda: sph.fragments(ctxf, dsf, link=1.01, d_remove=1.0, min_size=3),
                                         ctxf)
    frag = {"workload": "friends-of-friends of the fragmented body (%d particles, 10 damaged slabs, link 1.01 h)"
                        % fb.n,
            "ms": ms_g, "fragments": int(cnt.numel()), "value": fb.n / (ms_g * 1e-3), "unit": "particles/s",
            "phases_ms": ph_g}
    if with_oracle:
        sec, cores = oracle_time(lambda o: o.fof(fb.x, fb.h, fb.m, 3, b=1.01, d_remove=1.0, min_size=3, dmg=fb.dmg))
        frag["cpu_baseline"] = {"value": fb.n / sec, "unit": "particles/s", "cores": cores, "kind": "oracle",
                                "sample": "the same call on the host (%.1f s)" % sec}
    del dsf, lab, cnt, mass, ctxf

    # gravity/hydro decoupling (Sect. 6.3): the 2M-particle collapsing cloud,
    # steps that build a tree per evaluation against steps that reuse one
    # tree (and its pseudo-particles) over 4 steps
    cl = wl.cloud_collapse(seed=3, n=cloud_n)
    cctx = sph.Context(3, cl.n, max_neighbours=128, leaf_size=cl.params.leaf_size)
    dec = {"workload": "rotating cloud collapse, %d particles, Barnes-Hut theta %g, mixed precision" %
                       (cl.n, cl.params.theta)}
    for R in (0, 4):
        prm = replace(cl.params, precision="mixed", tree_reuse=R)
        dsc = sph.DeviceState(cl)
        sph.step(cctx, dsc, cl.materials, prm, 1, check=False)
        cctx.sync_status()
        cctx.profile(True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sph.step(cctx, dsc, cl.materials, prm, 2 * 4, check=False)  # two windows of 4 steps in one call
        b.record(stream)
        b.synchronize()
        ph = cctx.profile_read()
        cctx.profile(False)
        cctx.sync_status()
        dec["tree_reuse_%d" % R] = {"ms_per_step": a.elapsed_time(b) / 8,
                                    "phases_ms_per_step": {k: v[0] / 8 for k, v in ph.items() if v[1] > 0}}
        del dsc
    dec["speedup"] = dec["tree_reuse_0"]["ms_per_step"] / dec["tree_reuse_4"]["ms_per_step"]
    # the Barnes-Hut walk alone (sph_gravity on the initial cloud): its
    # interactions (device counters) and the FP32 rate they give, with 25 FP32
    # operations per interaction (difference of hi/lo positions 9, r^2 5,
    # softening 1, reciprocal square root 1, cube 2, mass 1, components 3,
    # accumulation 3) against the measured FMA peak
    prm = replace(cl.params, precision="mixed")
    dsc = sph.DeviceState(cl)
    sph.gravity(cctx, dsc, prm)
    cctx.sync_status()
    cctx.profile(True)
    sph.gravity(cctx, dsc, prm, check=False)
    ms_g = cctx.profile_read()["gravity"][0]  # the walk's own CUDA events (the call also builds a tree)
    gc = cctx.profile_counters()
    cctx.profile(False)
    cctx.sync_status()
    inter = gc["grav_nodes"] + gc["grav_terms"]
    fp32_peak = sph.measure_fma_peak("mixed")
    dec["gravity_walk"] = {
        "ms": ms_g, "nodes_per_particle": gc["grav_nodes"] / cl.n, "terms_per_particle": gc["grav_terms"] / cl.n,
        "interactions_per_s": inter / (ms_g * 1e-3), "flop_per_interaction": 25,
        "fp32_tflops": 25 * inter / (ms_g * 1e-3) / 1e12, "fp32_peak_tflops_measured": fp32_peak / 1e12,
        "fp32_frac": 25 * inter / (ms_g * 1e-3) / fp32_peak,
        "lane_use": inter / (32.0 * gc["grav_visits"]) if gc["grav_visits"] else None}
    del dsc
    del cctx

    # batched instances: the 256 impacts of uneven size in one concatenated
    # state, 4 steps per launch sequence, replayed from a captured CUDA graph
    # and launched directly
    bt = wl.batched_impacts(seed=5)
    bctx = sph.Context(3, bt.n, max_instances=bt.ninst, max_neighbours=128, leaf_size=bt.params.leaf_size)
    sph.fill_flaws(bctx, bt)
    # one tree per 4 steps (the window of one replay): 15.3 against 17.7 ms per
    # step with a tree per evaluation
    bprm = replace(bt.params, precision="mixed", tree_reuse=4)
    dsb = sph.DeviceState(bt)
    graph = sph.StepGraph(bctx, dsb, bt.materials, bprm, nsteps=4)
    graph.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gstream = graph.stream
    a.record(gstream)
    with torch.cuda.stream(gstream):
        for _ in range(3):
            graph.replay()
    b.record(gstream)
    b.synchronize()
    ms_graph = a.elapsed_time(b) / 12
    bctx.sync_status()
    del graph
    dsb = sph.DeviceState(bt)
    # the same steps as the graph's timed replays: steps 6..17 of the run (the
    # graph ran a warm-up step and one untimed replay of 4 before them)
    sph.step(bctx, dsb, bt.materials, bprm, 1, check=False)
    sph.step(bctx, dsb, bt.materials, bprm, 4, check=False)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    sph.step(bctx, dsb, bt.materials, bprm, 12, check=False)
    b.record(stream)
    b.synchronize()
    ms_plain = a.elapsed_time(b) / 12
    bctx.sync_status()
    batched = {"workload": "%d independent basalt impacts, %d particles in one state (targets 2k-50k log-uniform)" %
                           (bt.ninst, bt.n),
               "tree_reuse": bprm.tree_reuse, "ms_per_step_graph": ms_graph, "ms_per_step_launched": ms_plain,
               "value": bt.n / (ms_graph * 1e-3), "unit": "particle-updates/s"}
    del dsb, bctx, bt

    # adjoint of the right-hand side (FP64, damage off), 1M measured configuration
    ad = wl.measurement_1m(seed=21, n_side=100, damage=False)
    rng = np.random.default_rng(21)
    ad.u = rng.uniform(0.0, 6e6, ad.n)
    ad.S = rng.normal(0.0, 0.4 * ad.materials[0].Y0, (6, ad.n))
    aprm = replace(ad.params, alpha=1.0, beta=2.0, xsph=0.5, precision="fp64")
    actx = sph.Context(3, ad.n, max_neighbours=128, leaf_size=aprm.leaf_size)
    dsa = sph.DeviceState(ad)
    out = sph.rhs(actx, dsa, ad.materials, aprm, check=False)
    dbar = sph.alloc_derivs(dsa)
    for k in ("dxdt", "dv", "drho", "du", "dS"):
        dbar[k].normal_()
    sbar = dsa.zeros_like()
    pbar = torch.zeros((1, 1, 3), dtype=torch.float64, device="cuda")
    sph.rhs_adjoint(actx, dsa, ad.materials, aprm, dbar, sbar, pbar, check=False)
    adjoint = {"workload": "right-hand side and its adjoint (damage off), %d particles, measured configuration" %
                           ad.n}
    for prec in ("fp64", "mixed"):
        pp = replace(aprm, precision=prec)
        sph.rhs_adjoint(actx, dsa, ad.materials, pp, dbar, sbar, pbar, check=False)
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        for _ in range(3):
            sph.rhs(actx, dsa, ad.materials, pp, out=out, check=False)
        b.record(stream)
        for _ in range(3):
            sph.rhs_adjoint(actx, dsa, ad.materials, pp, dbar, sbar, pbar, check=False)
        c.record(stream)
        c.synchronize()
        actx.sync_status()
        adjoint["ms_rhs_" + prec] = a.elapsed_time(b) / 3
        adjoint["ms_adjoint_" + prec] = b.elapsed_time(c) / 3
    adjoint["adjoint_over_rhs_fp64"] = adjoint["ms_adjoint_fp64"] / adjoint["ms_rhs_fp64"]
    adjoint["adjoint_speedup_mixed_over_fp64"] = adjoint["ms_adjoint_fp64"] / adjoint["ms_adjoint_mixed"]
    del dsa, actx, out, dbar, sbar
    adjoint["rollout_256"] = adjoint_rollout(sph, wl, stream)
    return {"flaws": flaws, "fragments": frag, "decoupled_gravity": dec, "batched": batched, "adjoint": adjoint}


# ----------------------------------------------------------------------------
# CPU oracle as a baseline (the oracle as it stands, all host cores)
# ----------------------------------------------------------------------------
def host_steps(sph, ctx, ds, host, materials, prm, nsteps, stream):
    """nsteps predictor-corrector steps of a state that lives in pinned host
    memory (`host`: the fields of ds as pinned CPU tensors): every step uploads
    all its inputs and downloads its result (every field, since the step
    reorders the state along the tree).  The host link carries both
    directions at once: a field's upload for the next step starts as soon as
    its download has finished, while the other fields still come down.  The
    work is enqueued on `stream` (and two copy streams); returns without
    synchronising."""
    import torch
    outs = [k for k in ("x", "v", "rho", "u", "m", "h", "S", "dmg", "mat", "id") if host.get(k) is not None]
    cont = prm.tree_reuse > 0
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    got = {k: torch.cuda.Event() for k in outs}
    ready, done = torch.cuda.Event(), torch.cuda.Event()
    up.wait_stream(stream)
    for it in range(nsteps):
        with torch.cuda.stream(up):
            for k in outs:
                if it > 0:
                    up.wait_event(got[k])  # this field of the previous result is on the host
                getattr(ds, k).copy_(host[k], non_blocking=True)
            ready.record(up)
        stream.wait_event(ready)
        # each call continues the tree window of the last (the state it
        # uploads is the one the last call returned, which the call checks)
        sph.step(ctx, ds, materials, prm, 1, check=False, cont=cont and it > 0)
        done.record(stream)
        down.wait_event(done)
        with torch.cuda.stream(down):
            for k in outs:
                host[k].copy_(getattr(ds, k), non_blocking=True)
                got[k].record(down)
    stream.wait_stream(down)


def field_errors(sph, ctx, ps, prm):
    """Mixed against FP64 on the GPU, per field, on the measured state: one
    right-hand side each (max |mixed - fp64| over max |fp64| of the field, and
    the particles whose activated-flaw count differs), then one
    predictor-corrector step each on the same time step (the FP64 step's),
    compared by particle id relative to each field's change over the step."""
    import numpy as np
    from dataclasses import replace
    outs = {}
    for prec in ("mixed", "fp64"):
        ds = sph.DeviceState(ps)
        o = sph.rhs(ctx, ds, ps.materials, replace(prm, precision=prec))
        outs[prec] = {k: v.cpu().numpy() for k, v in o.items()}
        del ds, o
    rhs = {}
    for f in ("drho", "dv", "du", "dS", "dxdt", "p", "cs", "ddmg"):
        a, b = outs["mixed"][f].astype(np.float64), outs["fp64"][f].astype(np.float64)
        rhs[f] = float(np.abs(a - b).max() / (np.abs(b).max() + 1e-300))
    rhs["n_act_differs"] = int((outs["mixed"]["n_act"] != outs["fp64"]["n_act"]).sum())
    states = {}
    dt = None
    for prec in ("fp64", "mixed"):
        ds = sph.DeviceState(ps)
        p = replace(prm, precision=prec) if dt is None else replace(prm, precision=prec, dt_fixed=dt)
        d = sph.step(ctx, ds, ps.materials, p, 1)
        dt = float(d[0].item()) if dt is None else dt
        g = ds.to_numpy()
        order = np.argsort(g["id"])
        states[prec] = {k: g[k][..., order] for k in ("x", "v", "rho", "u", "S", "dmg")}
        del ds
    init = {"x": ps.x, "v": ps.v, "rho": ps.rho, "u": ps.u, "S": ps.S, "dmg": ps.dmg}
    step = {}
    for f in init:
        change = np.abs(states["fp64"][f] - init[f]).max() + 1e-300
        step[f] = float(np.abs(states["mixed"][f] - states["fp64"][f]).max() / change)
    return {"rhs_max_over_field_max": rhs, "step_max_over_field_change": step, "dt": dt,
            "what": "mixed vs FP64 GPU on the measured state: one right-hand side, and one step on the same dt"}


def reduce_max_ms(ms, dist, device):
    """The slowest rank's time: every rank runs its own replica, and the job
    takes as long as the slowest (max over ranks; NCCL on GPUs, gloo on CPU)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, units_per_rank, steps, ms):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return world * units_per_rank * steps / (ms * 1e-3)


def cpu_baseline(n_side, steps=1, repeats=3):
    """The oracle's predictor-corrector step on the host cores: one untimed
    warm-up call, then the median of `repeats` timed calls of `steps` steps."""
    import oracle
    from paper_1604_03290_gb300 import workloads as wl
    oracle.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    oracle.set_threads(cores)
    ps = wl.measurement_1m(seed=11, n_side=n_side)
    oracle.step(ps, ps.materials, ps.params, 1)
    ts = []
    for _ in range(max(repeats, 1)):
        t0 = time.perf_counter()
        oracle.step(ps, ps.materials, ps.params, steps)
        ts.append(time.perf_counter() - t0)
    dt = statistics.median(ts)
    return {"value": ps.n * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "same physics at %d^3 cube particles (%d particles), %d predictor-corrector step(s) per call, "
                      "median of %d calls after a warm-up call: %.2f s on %d host threads"
                      % (n_side, ps.n, steps, len(ts), dt, cores), "seconds": dt}


def run_reference(args, rank):
    if rank != 0:
        return
    base = cpu_baseline(args.cpu_side, steps=max(args.steps, 1), repeats=1)
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * base["seconds"] / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_cube_side": args.cpu_side},
            "cpu_baseline": {k: base[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import numpy as np
    import torch
    from dataclasses import replace

    from paper_1604_03290_gb300 import sph
    from paper_1604_03290_gb300 import workloads as wl

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ps = wl.measurement_1m(seed=11, n_side=args.n_side)
    n = ps.n
    prm = replace(ps.params, precision="mixed", tree_reuse=args.tree_reuse)
    ctx = sph.Context(3, n, max_neighbours=128, leaf_size=prm.leaf_size)
    sph.fill_flaws(ctx, ps)  # the Weibull flaws, drawn on the device (sph_flaws)
    stream = torch.cuda.current_stream()
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm_peak, peak_src = 6800.0, "fallback 6.8 TB/s"
    if os.path.exists(peaks_path):
        with open(peaks_path) as f:
            hbm_peak = float(json.load(f)["hbm_gbs"])
        peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)"
    if args.only_aux:
        if rank == 0:
            print(json.dumps({"next_rows": aux_rows(sph, wl, ctx, ps, stream, hbm_peak, cloud_n=args.cloud_n)}),
                  flush=True)
        return

    # mean partner count and flaw count for the byte model (outside timing)
    ds = sph.DeviceState(ps)
    out = sph.rhs(ctx, ds, ps.materials, prm)
    K = float(out["nnb"].double().mean().item())
    n_flaw = float(np.diff(ps.flaw_off).mean())
    del out

    # ---- device-resident throughput (mixed) ----
    ds = sph.DeviceState(ps)
    sph.step(ctx, ds, ps.materials, prm, args.warmup, check=False)
    ctx.sync_status()
    clocks = ClockSampler(local)
    barrier()
    if rank == 0:
        clocks.start()
        time.sleep(0.3)
    ctx.profile(True)
    l0 = sph.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    # the K steps in one call (a tree serves tree_reuse consecutive steps)
    sph.step(ctx, ds, ps.materials, prm, args.steps, check=False)
    e1.record(stream)
    e1.synchronize()
    launches = sph.launch_count() - l0
    phases = ctx.profile_read()
    ctrs = ctx.profile_counters()
    ctx.profile(False)
    ms = e0.elapsed_time(e1)
    clk = clocks.stop() if rank == 0 else None
    barrier()
    ctx.sync_status()
    ms = reduce_max_ms(ms, dist, "cuda")
    value = replica_value(world, n, args.steps, ms)

    # ---- rooflines ----
    # The partner walk and the neighbour passes are bound by instruction issue
    # (latency and ALU work of irregular gathers and an irregular tree walk):
    # their roofline is warp instructions issued per second against SMs x 4
    # issue slots x the SM clock seen under load.  Each is also reported
    # against HBM with its algorithmic bytes (each array once).  Launch times
    # are the library's CUDA events on the launching stream over the timed
    # region.
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
    issue_peak = nsm * ISSUE_SLOTS_PER_SM * sm_mhz * 1e6 / 1e9  # G warp-instructions / s

    def kernel_roof(phase):
        calls = phases.get(phase, (0.0, 0))
        if calls[1] == 0:
            return None
        launch_ms = calls[0] / calls[1]
        ab = algorithmic_bytes(phase, K, n_flaw) * n
        r = {"avg_launch_ms": launch_ms,
             "hbm": {"achieved": ab / (launch_ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                     "frac": ab / (launch_ms * 1e-3) / 1e9 / hbm_peak,
                     "bytes_per_particle": algorithmic_bytes(phase, K, n_flaw)}}
        c = ncu_figures(phase)
        r["ncu_current"] = c is not None
        if c:
            ginst = c["inst"] * n / (launch_ms * 1e-3) / 1e9
            r["issue"] = {"achieved": ginst, "peak": issue_peak, "unit": "G warp-instructions/s",
                          "frac": ginst / issue_peak, "inst_per_particle_ncu": c["inst"]}
            r["dram_bytes_ncu"] = c["dram"] * n
            r["fp32_pipe_frac_ncu"] = c["fp32_pipe"]
            r["l1_throughput_frac_ncu"] = c["l1"]
        return r

    kr = {p: kernel_roof(p) for p in ("partners", "refine", "passA", "passB")}
    timed = {p: phases[p][0] for p in kr if kr[p] is not None}
    dom = max(timed, key=timed.get) if timed else "partners"
    d = kr[dom]
    if "issue" in d:
        roof = {"bound": "alu", "kernel": dom, "achieved": d["issue"]["achieved"], "peak": issue_peak,
                "unit": "G warp-instructions/s", "frac": d["issue"]["frac"],
                "traffic": d.get("dram_bytes_ncu"),
                "peak_source": "%d SMs x %d issue slots x %.0f MHz (median SM clock under load)" %
                               (nsm, ISSUE_SLOTS_PER_SM, sm_mhz),
                "avg_launch_ms": d["avg_launch_ms"], "hbm_frac_algorithmic": d["hbm"]["frac"],
                "fp32_pipe_frac_ncu": d.get("fp32_pipe_frac_ncu")}
    else:
        roof = {"bound": "hbm", "kernel": dom, "achieved": d["hbm"]["achieved"], "peak": hbm_peak, "unit": "GB/s",
                "frac": d["hbm"]["frac"], "traffic": d.get("dram_bytes_ncu"), "peak_source": peak_src,
                "avg_launch_ms": d["avg_launch_ms"]}
    roof["mean_partners"] = K
    walks = phases.get("reorder", (0.0, 0))[1]  # one walk over all particles per tree build
    if walks:
        roof["partner_walk_counters"] = {
            "candidates_tested_per_particle": ctrs["walk_tests"] / (walks * n),
            "partners_per_particle": ctrs["walk_partners"] / (walks * n), "walks": walks}
    roof["kernels"] = kr
    total_ms = sum(v[0] for v in phases.values())
    phase_report = {p: {"ms_per_step": v[0] / args.steps, "share": v[0] / total_ms if total_ms else None,
                        "launch_ms": v[0] / v[1] if v[1] else None}
                    for p, v in phases.items() if v[1] > 0}

    # ---- FP64 step on the same workload ----
    fp64 = None
    if args.fp64_steps > 0:
        prm64 = replace(prm, precision="fp64")
        ds64 = sph.DeviceState(ps)
        sph.step(ctx, ds64, ps.materials, prm64, 1, check=False)
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        sph.step(ctx, ds64, ps.materials, prm64, args.fp64_steps, check=False)
        f1.record(stream)
        f1.synchronize()
        ctx.sync_status()
        ms64 = f0.elapsed_time(f1) / args.fp64_steps
        fp64 = {"value": n / (ms64 * 1e-3), "ms_per_step": ms64, "unit": UNIT}
        del ds64

    # ---- end to end through the C ABI with host buffers ----
    host = {k: (None if v is None else v.detach().cpu().pin_memory()) for k, v in
            {"x": ds.x, "v": ds.v, "rho": ds.rho, "u": ds.u, "m": ds.m, "h": ds.h, "S": ds.S, "dmg": ds.dmg,
             "mat": ds.mat, "id": ds.id}.items()}
    h2d = sum(t.numel() * t.element_size() for t in host.values() if t is not None)
    # the step reorders every field along the tree, so the result is all of them
    d2h = h2d
    e2e_steps = max(3, args.steps // 3)
    barrier()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    host_steps(sph, ctx, ds, host, ps.materials, prm, e2e_steps, stream)
    g1.record(stream)
    g1.synchronize()
    ms_e2e = g0.elapsed_time(g1)
    ms_e2e = reduce_max_ms(ms_e2e, dist, "cuda")
    e2e = {"value": replica_value(world, n, e2e_steps, ms_e2e), "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}

    ferr = field_errors(sph, ctx, ps, prm) if rank == 0 else None

    aux = (aux_rows(sph, wl, ctx, ps, stream, hbm_peak, cloud_n=args.cloud_n,
                    with_oracle=rank == 0 and not args.no_cpu) if not args.no_aux else None)

    cpu = None
    if rank == 0 and not args.no_cpu:
        b = cpu_baseline(args.cpu_side, steps=1)
        cpu = {k: b[k] for k in ("value", "unit", "cores", "kind", "sample")}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32 pair/f64 state (mixed)", "data": "synthetic",
                "config": {"workload": WORKLOAD, "n_particles": n, "mean_partners": K,
                           "tree_reuse": args.tree_reuse,
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "l2": "inputs larger than L2 (state %.0f MB, partner lists %.0f MB)" %
                                 (144 * n / 1e6, 4 * K * n / 1e6)},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "fp64": fp64,
                "speedup_mixed_over_fp64": (value / world / fp64["value"]) if fp64 else None,
                "field_errors": ferr,
                "phases": phase_report, "next_rows": aux}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
