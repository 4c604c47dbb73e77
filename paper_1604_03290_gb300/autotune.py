"""Autotuner for the launch shapes and walk granularity of a context.

Times one right-hand side per candidate (CUDA events per phase, on the call's
stream) on the caller's own workload and keeps the fastest.  Every candidate
gives bit-identical results: the partner lists come out in ascending slot order
whatever the walk granularity, the sums are per thread, and the tree leaf size
is only searched when gravity is off (with gravity it changes which nodes the
Barnes-Hut walk accepts).  Results are cached in a JSON file keyed by device,
dimension, physics flags and a particle-count bucket.
"""
from __future__ import annotations

import itertools
import json
import math
import os
from dataclasses import replace

import torch

from . import sph

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "sph_gb300_tuning.json")


def _key(ds, params):
    name = torch.cuda.get_device_name()
    bucket = int(round(math.log2(max(ds.n, 1))))
    flags = "g%d_d%d_s%d_as%d" % (int(params.gravity), int(params.density_sum), int(ds.S is not None),
                                  int(params.eps_s > 0))
    return "%s|dim%d|%s|n2^%d|%s" % (name, ds.dim, flags, bucket, params.precision)


def _time_rhs(ctx, ds, materials, params, reps=2):
    sph.rhs(ctx, ds, materials, params, check=False)
    torch.cuda.synchronize()
    ctx.profile(True)
    for _ in range(reps):
        sph.rhs(ctx, ds, materials, params, check=False)
    ph = ctx.profile_read()
    ctx.profile(False)
    return sum(v[0] for v in ph.values()) / reps


def candidates(params):
    leaves = [params.leaf_size] if params.gravity else [8, 16, 32]
    return [dict(leaf_size=L, walk_leaf=w, walk_blocks_per_sm=b, pass_threads=t)
            for L, w, b, t in itertools.product(leaves, (32, 64, 128, 256), (8, 12, 16, 24), (64, 128))]


def tune(ctx: sph.Context, ds: sph.DeviceState, materials, params, cache_path=DEFAULT_CACHE, use_cache=True,
         cands=None):
    """Returns (params with the chosen leaf_size, tuning dict, ms per RHS) and
    applies the tuning to ``ctx``."""
    key = _key(ds, params)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        best = cache[key]
    else:
        best, best_ms = None, float("inf")
        for c in (cands or candidates(params)):
            ctx.set_tuning(walk_leaf=c["walk_leaf"], walk_blocks_per_sm=c["walk_blocks_per_sm"],
                           pass_threads=c["pass_threads"])
            ms = _time_rhs(ctx, ds, materials, replace(params, leaf_size=c["leaf_size"]))
            if ms < best_ms:
                best, best_ms = dict(c, ms=ms), ms
        ctx.sync_status()
        if cache_path:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            cache[key] = best
            tmp = cache_path + ".%d.tmp" % os.getpid()
            json.dump(cache, open(tmp, "w"), indent=1)
            os.replace(tmp, cache_path)
    ctx.set_tuning(walk_leaf=best["walk_leaf"], walk_blocks_per_sm=best["walk_blocks_per_sm"],
                   pass_threads=best["pass_threads"])
    return replace(params, leaf_size=best["leaf_size"]), best, best.get("ms")
