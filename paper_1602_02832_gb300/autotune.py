"""Autotuner for the force work decomposition: i tile size (tile_i, particles
per static tile), list part length (tile_j) and work-item cost target
(work_item).

For a given workload (a particle set and its tree settings) every candidate
runs the same short stretch of the real tree loop — start-up, a warm-up tree
interval, then timed intervals of block steps plus rebuilds through the
persistent batched loop — and the candidate with the most interactions per
second wins.  Results are kept in a JSON cache keyed by device, precision,
N (rounded to a power of two), theta and n_crit.  Tuning runs outside any
timed region.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from . import HH_FP64, HH_MIXED, Batch, Context, hh_config_default, hh_tree_build

CANDIDATES = {
    HH_FP64: [dict(tile_i=ti, tile_j=tj, work_item=0) for ti in (32, 16) for tj in (128, 256, 512)],
    HH_MIXED: [dict(tile_i=ti, tile_j=tj, work_item=0) for ti in (32, 16) for tj in (256, 512, 1024)],
}

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _key(device_name, precision, n, theta, n_crit):
    return f"{device_name}|{'mixed' if precision == HH_MIXED else 'fp64'}|n2^{round(math.log2(max(n, 2)))}|" \
           f"theta{theta}|ncrit{n_crit}"


def _run_candidate(x, v, m, base, cand, intervals, warm):
    n = len(m)
    cfg = hh_config_default()
    for f, _ in base._fields_:
        setattr(cfg, f, getattr(base, f))
    for k, val in cand.items():
        setattr(cfg, k, val)
    z = np.zeros((3, n))
    T = hh_tree_build(x.T, v.T, z, z, m, leaf=cfg.leaf, n_crit=cfg.n_crit, theta=cfg.theta)
    dtt = cfg.dt_tree
    with Context(cfg, n, 2 * n, int(2 * len(T.idx)) + 1024, 2 * T.n_groups + 64) as ctx, \
            Batch(cfg.precision, max_sims=1, max_steps=4096) as b:
        ctx.hh_load_particles(np.ascontiguousarray(x.T), np.ascontiguousarray(v.T), m)
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
        c0 = ctx.hh_get_counters()["interactions"]
        w0 = time.perf_counter()
        for _ in range(intervals):
            interval()
        dt = time.perf_counter() - w0
        return (ctx.hh_get_counters()["interactions"] - c0) / dt


def tune(x, v, m, base_cfg, intervals=1, warm=1, use_cache=True, device_name=None):
    """Returns (best candidate dict, table of (candidate, interactions/s))."""
    if device_name is None:
        try:
            import torch
            device_name = torch.cuda.get_device_name(0)
        except Exception:
            device_name = "cuda"
    key = _key(device_name, base_cfg.precision, len(m), round(base_cfg.theta, 3), base_cfg.n_crit)
    cache = {}
    if use_cache and os.path.exists(_CACHE):
        try:
            cache = json.load(open(_CACHE))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return cache[key]["best"], cache[key]["table"]
    table = []
    for cand in CANDIDATES[base_cfg.precision]:
        rate = _run_candidate(x, v, m, base_cfg, cand, intervals, warm)
        table.append((cand, rate))
    best = max(table, key=lambda r: r[1])[0]
    if use_cache:
        cache[key] = {"best": best, "table": table}
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        tmp = _CACHE + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, _CACHE)
    return best, table
