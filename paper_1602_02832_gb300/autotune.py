"""Autotuner for the group size and the force work decomposition: n_crit
(particles per group sharing one list: the paper sets it to the value that
minimises the total computing time, Section 2), i tile size (tile_i,
particles per static tile), list part length (tile_j), work-item cost
target (work_item) and the step size from which it applies (work_split).

For a given workload (a particle set and its tree settings) every candidate
runs the same short stretch of the real tree loop — start-up, a warm-up tree
interval, then timed intervals of block steps plus rebuilds through the
persistent batched loop — and the candidate that advances the simulation
fastest (particle steps per second, i.e. shortest time to solution; the
interaction count itself grows with n_crit) wins.  Results are kept in a JSON
cache keyed by device, precision, N (rounded to a power of two) and theta.
Tuning runs outside any timed region.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from . import HH_FP64, HH_MIXED, Batch, Context, hh_config_default, hh_tree_build

# work_item > 0 with work_split > 0: equal-cost list parts only in block steps
# with at least work_split active particles (the batched loop; per-step
# profiles of the N = 65536 run: the force phase of large steps 2-8% faster,
# small steps unchanged).  tile_j_small: short parts in steps with at most 16
# due particles (their force phase 2-3% shorter in all).
CANDIDATES = {
    HH_FP64: [dict(n_crit=nc, tile_i=ti, tile_j=tj, work_item=0, work_split=0)
              for nc in (64, 256) for ti in (32, 16, 8) for tj in (128, 256, 512)]
             + [dict(n_crit=nc, tile_i=ti, tile_j=256, work_item=0, work_split=0) for nc in (128, 1024) for ti in (16, 8)]
             + [dict(n_crit=64, tile_i=ti, tile_j=256, work_item=wk, work_split=2048)
                for ti in (16, 8) for wk in (1024, 2048)]
             + [dict(n_crit=64, tile_i=8, tile_j=256, work_item=2048, work_split=2048, tile_j_small=sm)
                for sm in (32, 64)],
    HH_MIXED: [dict(n_crit=nc, tile_i=ti, tile_j=tj, work_item=0, work_split=0)
               for nc in (64, 256) for ti in (32, 16) for tj in (256, 512, 1024)]
              + [dict(n_crit=nc, tile_i=32, tile_j=512, work_item=0, work_split=0) for nc in (128, 1024)]
              + [dict(n_crit=nc, tile_i=32, tile_j=512, work_item=wk, work_split=513)
                 for nc in (64, 128) for wk in (8192, 16384)]
              + [dict(n_crit=nc, tile_i=32, tile_j=512, work_item=8192, work_split=513, tile_j_small=128)
                 for nc in (64, 128)],
}

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _key(device_name, precision, n, theta, rebuild_device, order=0):
    return f"{device_name}|{'mixed' if precision == HH_MIXED else 'fp64'}|n2^{round(math.log2(max(n, 2)))}|" \
           f"theta{theta}|{'dev' if rebuild_device else 'host'}|order{order}"


def _run_candidate(x, v, m, base, cand, intervals, warm, rebuild_device):
    n = len(m)
    cfg = hh_config_default()
    for f, _ in base._fields_:
        setattr(cfg, f, getattr(base, f))
    for k, val in cand.items():
        setattr(cfg, k, val)
    z = np.zeros((3, n))
    T = hh_tree_build(x.T, v.T, z, z, m, leaf=cfg.leaf, n_crit=cfg.n_crit, theta=cfg.theta, order=cfg.order)
    dtt = cfg.dt_tree
    with Context(cfg, n, 2 * n, int(2 * len(T.idx)) + 1024, 2 * T.n_groups + 64) as ctx, \
            Batch(cfg.precision, max_sims=1, max_steps=4096) as b:
        ctx.hh_load_particles(np.ascontiguousarray(x.T), np.ascontiguousarray(v.T), m)
        ctx.hh_set_rebuild_device(rebuild_device)
        ctx.hh_run(0.0, 0.0)
        t = 0.0

        def interval():
            nonlocal t
            while True:
                _, tn, _ = b.hh_batch_run([ctx], [t + dtt])
                if tn[0] > t + dtt:
                    break
            ctx.hh_rebuild(t + dtt)
            t += dtt

        for _ in range(warm):
            interval()
        c0 = ctx.hh_get_counters()
        w0 = time.perf_counter()
        for _ in range(intervals):
            interval()
        dt = time.perf_counter() - w0
        c1 = ctx.hh_get_counters()
        return (c1["particle_steps"] - c0["particle_steps"]) / dt, (c1["interactions"] - c0["interactions"]) / dt


def tune(x, v, m, base_cfg, intervals=1, warm=1, use_cache=True, device_name=None, rebuild_device=False):
    """Returns (best candidate dict, table of (candidate, particle steps/s, interactions/s)).
    rebuild_device selects where the tuning runs rebuild the tree (the cost of
    a rebuild depends on n_crit, so the choice is part of the cache key)."""
    if device_name is None:
        try:
            import torch
            device_name = torch.cuda.get_device_name(0)
        except Exception:
            device_name = "cuda"
    key = _key(device_name, base_cfg.precision, len(m), round(base_cfg.theta, 3), rebuild_device, base_cfg.order)
    cache = {}
    if use_cache and os.path.exists(_CACHE):
        try:
            with open(_CACHE) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return cache[key]["best"], cache[key]["table"]
    table = []
    for cand in CANDIDATES[base_cfg.precision]:
        steps_rate, int_rate = _run_candidate(x, v, m, base_cfg, cand, intervals, warm, rebuild_device)
        table.append((cand, steps_rate, int_rate))
    best = max(table, key=lambda r: r[1])[0]
    if use_cache:
        cache[key] = {"best": best, "table": table}
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        tmp = _CACHE + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, _CACHE)
    return best, table
