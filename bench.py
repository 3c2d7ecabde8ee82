#!/usr/bin/env python
"""Benchmark of the list-driven 4th-order Hermite path (libhh) on GB300.

Workload (default): the full plain run — N = 65536 Plummer sphere (standard
units, equal masses, seed = rank), 4th-order Hermite with power-of-two block
steps (Aarseth eta = 0.02, dt in [2^-30, 2^-6]: the requested 2^-3 is clamped
to dt_tree because the tree loop caps every step at the rebuild interval),
tree and lists rebuilt every dt_tree = 1/64, theta = 0.5, eps = 1e-4, FP64.

One step = one tree interval dt_tree: all block steps of the interval on the
device (persistent batched loop, or CUDA graph replays of predict / force /
correct with --loop graph) followed by the tree rebuild: on the device by
default (Morton keys, radix sort, cells, node records, groups and lists built
by the library's kernels without the state leaving the GPU); --rebuild host
takes the state to the host, runs the library's host tree builder and
uploads particles, nodes and lists.  Warm-up intervals start at t = 0; the timed
intervals follow.  L2 is flushed (256 MB write) before each timed interval.

value = interactions / time (interactions = sum over particle steps of the
list length minus self), timed with CUDA events on the context's stream; the
same line reports the mixed-precision form on the same workload, block steps
per second, the roofline of the force kernel against measured FMA peaks, an
end-to-end figure through host buffers, and the FP64 oracle as CPU baseline.

--impl reference times the FP64 CPU oracle on the same workload (a bounded
sample per step) on the host cores.
"""
from __future__ import annotations

import argparse
import ctypes as C
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

FLOP_PER_INT = 60
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one k_batch
# launch, plain FP64, one 1/64 interval of the N = 65536 run, from one ncu
# capture of that launch.  It holds only for the kernel sources it was taken
# with (their digest below) and for the tile shape it was taken with: when
# either differs, the line reports null.
TRAFFIC_FP64 = {"bytes": 85334528 + 55208704, "sources_sha16": "40d38e1904af32d4",
                "shape": {"n_crit": 64, "tile_i": 8, "tile_j": 256, "work_item": 2048, "work_split": 2048,
                          "tile_j_small": 64},
                "capture": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none "
                           "-k regex:k_batch -s 1 -c 1 on bench.py --steps 1 --warmup 1 --no-mixed "
                           "--no-autotune --n-crit 64 --tile-i 8 --tile-j 256 --work-item 2048 "
                           "--work-split 2048 --tile-j-small 64 --ensemble 0 --serve-seconds 0 "
                           "--no-cpu-baseline --no-config1 --no-config3"}
KERNEL_SOURCES = ("paper_1602_02832_gb300/csrc/hh_batch.cu", "paper_1602_02832_gb300/csrc/hh_kernels.cuh")
METRIC = "interactions/s & equiv. Tflops (60 flop/int); block-steps/s, p50/p99 latency vs plain"
CPU_SAMPLE_T = 1.0 / 256  # reference arm, per step: the first quarter of the first timed interval
CPU_BASELINE_T = 4.0 / 64  # cpu_baseline leg: the first four timed intervals (about 12 s on 16 cores)


def _sources_sha16():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(shape):
    """Captured DRAM bytes per launch if the kernel sources and the tile shape
    are those of the capture, else None."""
    if (TRAFFIC_FP64["bytes"] and TRAFFIC_FP64["sources_sha16"] == _sources_sha16()
            and shape == TRAFFIC_FP64["shape"]):
        return TRAFFIC_FP64["bytes"]
    return None


SHAPE_KEYS = ("n_crit", "tile_i", "tile_j", "work_item", "work_split", "tile_j_small")


def _args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=8)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="hh", choices=["hh", "reference"])
    p.add_argument("--n", type=int, default=65536)
    p.add_argument("--n-crit", type=int, default=64, help="group size when the autotuner is off")
    p.add_argument("--theta", type=float, default=0.5)
    p.add_argument("--tile-i", type=int, default=0, help="particles per i tile, both forms (0: tuned default)")
    p.add_argument("--tile-j", type=int, default=0, help="list part length of the plain FP64 form (0: tuned default)")
    p.add_argument("--tile-j-mixed", type=int, default=0, help="list part length of the mixed form (0: tuned default)")
    p.add_argument("--work-item", type=int, default=0, help="interactions per work item, plain form (0: default)")
    p.add_argument("--work-item-mixed", type=int, default=0, help="interactions per work item, mixed form (0: default)")
    p.add_argument("--work-split", type=int, default=0,
                   help="active particles from which work items apply, plain form (0: every step)")
    p.add_argument("--work-split-mixed", type=int, default=0,
                   help="active particles from which work items apply, mixed form (0: every step)")
    p.add_argument("--tile-j-small", type=int, default=0,
                   help="list part length of block steps with at most 16 due particles, plain form (0: tile_j)")
    p.add_argument("--tile-j-small-mixed", type=int, default=0,
                   help="list part length of block steps with at most 16 due particles, mixed form (0: tile_j)")
    p.add_argument("--no-mixed", action="store_true")
    p.add_argument("--mixed-only", action="store_true", help="run only the mixed form (profiling aid)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--ensemble", type=int, default=256, help="clusters in the batched-ensemble measurement (0: skip)")
    p.add_argument("--ensemble-t-end", type=float, default=0.5,
                   help="end time of every ensemble cluster (a multiple of dt_tree = 1/64)")
    p.add_argument("--serve-seconds", type=float, default=20.0, help="wall time of the serving measurement (0: skip)")
    p.add_argument("--batch-work-item", type=int, default=8192,
                   help="equal-cost work items (interactions) of the ensemble and serving runs, mixed form (0: off); "
                        "with many simulations per launch the queue stays full, so balance pays in every step")
    p.add_argument("--batch-work-split", type=int, default=0,
                   help="active particles from which those work items apply (0: every step)")
    p.add_argument("--serve-sustained-rate", type=float, default=4.0,
                   help="arrival rate (1/s) of the second serving measurement, a load the server keeps up with "
                        "(0: skip)")
    p.add_argument("--serve-sustained-seconds", type=float, default=40.0,
                   help="wall time of the second serving measurement")
    p.add_argument("--serve-launch-particles", type=int, default=1 << 21,
                   help="particles advanced per launch in both serving measurements (latency control; 0: no cap)")
    p.add_argument("--no-autotune", action="store_true", help="skip the tile-shape autotuner (use the defaults)")
    p.add_argument("--order", default="morton", choices=["morton", "hilbert"],
                   help="order of particles and nodes in the tree (Peano-Hilbert is the paper's)")
    p.add_argument("--rebuild", default="auto", choices=["auto", "device", "host"],
                   help="where the tree, groups and lists are rebuilt every dt_tree (auto: a lone simulation "
                        "on the device from N = 2048 and on the host below, where one device build is bound by "
                        "launch latency; the ensemble and serving servers on the device, in batched builds)")
    p.add_argument("--loop", default="persistent", choices=["persistent", "graph"],
                   help="block-step loop: one persistent cooperative kernel per interval, or CUDA-graph replays")
    p.add_argument("--no-config1", action="store_true",
                   help="skip the N = 4096 single force evaluation (direct sum and tree lists)")
    p.add_argument("--no-config3", action="store_true",
                   help="skip the N = 2^20 Plummer-Salpeter mixed-precision run to t = 0.125")
    return p.parse_args(argv)


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _cfg(hh, prec, a):
    c = hh.hh_config_default()
    c.eps2 = 1e-8
    c.eta = 0.02
    c.eta_s = 0.01
    c.dt_min = 2.0 ** -30
    c.dt_max = 2.0 ** -6
    c.dt_tree = 2.0 ** -6
    c.theta = a.theta
    c.leaf = 8
    c.n_crit = a.n_crit
    c.precision = prec
    c.tile_i = a.tile_i or 0
    c.tile_j = (a.tile_j if prec == hh.HH_FP64 else a.tile_j_mixed) or 0
    c.work_item = (a.work_item if prec == hh.HH_FP64 else a.work_item_mixed) or 0
    c.work_split = (a.work_split if prec == hh.HH_FP64 else a.work_split_mixed) or 0
    c.tile_j_small = (a.tile_j_small if prec == hh.HH_FP64 else a.tile_j_small_mixed) or 0
    c.order = hh.HH_ORDER_HILBERT if a.order == "hilbert" else hh.HH_ORDER_MORTON
    return c


def _on_device(a, n):
    from paper_1602_02832_gb300 import serve

    return a.rebuild == "device" or (a.rebuild == "auto" and n >= serve.AUTO_DEVICE_MIN_N)


def _server_rebuild(a):
    return "auto" if a.rebuild == "auto" else a.rebuild == "device"


def _workload(a):
    return (f"Plummer N={a.n}, 4th-order Hermite, power-of-two block steps (eta=0.02, dt in [2^-30, 2^-6]), "
            f"tree/lists rebuilt every dt_tree=1/64, theta={a.theta}, leaf 8, n_crit from the autotuner "
            f"(time to solution; {a.n_crit} without it), eps=1e-4; "
            f"one step = one dt_tree interval")


class Clocks:
    """nvidia-smi sampler (200 ms) running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [u.strip() for u in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks(hh_dir, device=0):
    """Measured FMA peaks (TFLOP/s) from libhh_peaks.so, plus the measured HBM / bf16 figures (MEASURED_PEAKS.json)."""
    out = {}
    lib = C.CDLL(os.path.join(hh_dir, "libhh_peaks.so"))
    lib.hh_fma_peak.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]
    for name, fp64, iters in (("fp32_tflops", 0, 200000), ("fp64_tflops", 1, 20000)):
        best = 0.0
        for _ in range(3):
            v = C.c_double()
            if lib.hh_fma_peak(device, fp64, iters, C.byref(v)) == 0:
                best = max(best, v.value)
        out[name] = best
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        out["hbm_gbs"] = mp.get("hbm_gbs")
        out["bf16_tflops"] = mp.get("bf16_tflops")
    except (OSError, ValueError):
        out["hbm_gbs"] = None
    return out


class _Loop:
    """Advances one context to a stop time with the chosen block-step loop and
    accumulates the force-kernel (or force-phase) time while enabled."""

    def __init__(self, hh, ctx, prec, kind):
        self.ctx, self.kind = ctx, kind
        self.batch = hh.Batch(prec, max_sims=1, max_steps=4096) if kind == "persistent" else None
        self.force_ms = 0.0
        self.force_launches = 0
        self.timing = False
        self.step_us = []
        self.phase_ms = [0.0, 0.0, 0.0]

    def enable(self, on):
        self.timing = on
        if self.kind == "graph":
            if on:
                self.ctx.hh_force_timing(1)
            else:
                self.force_ms, self.force_launches = self.ctx.hh_force_timing(0)

    def advance(self, t_end):
        if self.kind == "graph":
            self.ctx.hh_advance(t_end)
            return
        while True:
            steps, tn, us = self.batch.hh_batch_run([self.ctx], [t_end])
            if self.timing:
                ph = self.batch.last_phase_us
                self.force_ms += float(ph[:, 1].sum()) * 1e-3
                self.force_launches += int(steps)
                self.step_us.extend(us.tolist())
                for q in range(3):
                    self.phase_ms[q] += float(ph[:, q].sum()) * 1e-3
            if tn[0] > t_end:
                return

    def close(self):
        if self.batch:
            self.batch.close()


def reduce_over_ranks(sums, maxes, device, world):
    """Whole-job aggregation of independent replicas: work counts are summed
    and times take the maximum over ranks (the slowest rank bounds the job).
    No data-path collective: only these scalars cross ranks."""
    import torch

    t_sum = torch.tensor(sums, dtype=torch.float64, device=device)
    t_max = torch.tensor(maxes, dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t_sum, op=dist.ReduceOp.SUM)
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    return t_sum.tolist(), t_max.tolist()


def _tuned(hh, a, prec, seed):
    """Tile shape for this workload from the autotuner (outside the timed region)."""
    if a.no_autotune or a.tile_j or a.tile_j_mixed or a.tile_i:
        return {}, None
    import synth
    from paper_1602_02832_gb300 import autotune

    x, v, m = synth.plummer(a.n, seed)
    best, table = autotune.tune(x, v, m, _cfg(hh, prec, a), intervals=1, warm=1,
                                rebuild_device=_on_device(a, a.n))
    return best, [{"config": c, "particle_steps_per_s": ps, "interactions_per_s": r} for c, ps, r in table]


def _state_in_input_order(ctx, m, t):
    """The context's particle state (x, v, a, jerk [n, 3], dt [n]) in the order
    of the input arrays, with the masses m and time t."""
    import numpy as np

    st = ctx.hh_get_state()
    ids = ctx.hh_get_ids()
    n = len(m)
    out = {"m": m, "t": t}
    for k in ("x", "v", "a", "jk"):
        u = np.zeros((n, 3))
        u[ids] = st[k].T
        out[k] = u
    dt = np.zeros(n)
    dt[ids] = st["dt"]
    out["dt"] = dt
    return out


def _run_form(hh, torch, a, prec, seed, steps, warmup, flush, e2e_steps=0, over=None, keep_state=False):
    import numpy as np
    import synth

    x, v, m = synth.plummer(a.n, seed)
    cfg = _cfg(hh, prec, a)
    for k, val in (over or {}).items():
        setattr(cfg, k, val)
    z = np.zeros((3, a.n))
    T0 = hh.hh_tree_build(x.T, v.T, z, z, m, leaf=8, n_crit=cfg.n_crit, theta=a.theta)
    nj_max = 2 * a.n
    list_max = int(len(T0.idx) * 2) + 1024
    groups_max = int(T0.n_groups * 2) + 64
    ctx = hh.Context(cfg, a.n, nj_max, list_max, groups_max)
    stream = torch.cuda.Stream()
    ctx.hh_set_stream(stream.cuda_stream)
    dtt = cfg.dt_tree
    shape = {k: int(getattr(cfg, k)) for k in SHAPE_KEYS}
    ctx.hh_load_particles(x.T, v.T, m)
    ctx.hh_set_rebuild_device(_on_device(a, a.n))
    ctx.hh_run(0.0, 0.0)  # rebuild, initial forces, rebuild with node derivatives, initial steps
    loop = _Loop(hh, ctx, prec, a.loop)
    t = 0.0
    for _ in range(warmup):
        loop.advance(t + dtt)
        ctx.hh_rebuild(t + dtt)
        t += dtt
    # the synchronised state at the start of the timed window (the CPU
    # baseline resumes the oracle from it, so both time the same work)
    warm_state = _state_in_input_order(ctx, m, t) if keep_state else None
    c0 = ctx.hh_get_counters()
    h0 = ctx.hh_get_tile_histogram()
    l0 = hh.hh_kernel_launches()
    loop.enable(True)
    times = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        loop.advance(t + dtt)
        ctx.hh_rebuild(t + dtt)
        e1.record(stream)
        t += dtt
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    loop.enable(False)
    force_ms, force_launches = loop.force_ms, loop.force_launches
    launches = hh.hh_kernel_launches() - l0
    c1 = ctx.hh_get_counters()
    hist = (ctx.hh_get_tile_histogram() - h0).tolist()
    res = {
        "ms": sum(times), "step_ms": times,
        "interactions": c1["interactions"] - c0["interactions"],
        "block_steps": c1["block_steps"] - c0["block_steps"],
        "particle_steps": c1["particle_steps"] - c0["particle_steps"],
        "force_ms": force_ms, "force_launches": force_launches, "gpu_launches": launches, "t_end": t,
        "n_i_hist": hist, "warm_state": warm_state, "shape": shape,
    }
    if e2e_steps:
        # end to end through host buffers: upload the step's particle state,
        # run the interval, read the state back (pinned host copies)
        st = ctx.hh_get_state()
        n = a.n
        mm = np.ascontiguousarray(m[ctx.hh_get_ids()])
        bi = (4 * 3 * n + 2 * n) * 8 + n * 8
        bo = (4 * 3 * n + 2 * n) * 8
        c2 = ctx.hh_get_counters()
        e2e_ms = 0.0
        for _ in range(e2e_steps):
            torch.cuda.synchronize()
            w0 = time.perf_counter()
            ctx.hh_set_j(0, st["x"], st["v"], st["a"], st["jk"], mm, st["t"])
            ctx.hh_set_dt(st["dt"])
            loop.advance(t + dtt)
            ctx.hh_rebuild(t + dtt)
            st = ctx.hh_get_state()
            mm = np.ascontiguousarray(m[ctx.hh_get_ids()])
            e2e_ms += (time.perf_counter() - w0) * 1e3
            t += dtt
        c3 = ctx.hh_get_counters()
        res["e2e"] = {"ms": e2e_ms, "interactions": c3["interactions"] - c2["interactions"], "bi": bi, "bo": bo,
                      "steps": e2e_steps}
    res["step_us"] = loop.step_us
    res["phase_ms"] = loop.phase_ms
    loop.close()
    ctx.close()
    return res


def _ensemble(hh, a):
    """Batched form: 256 independent Plummer clusters, N log-uniform in
    [1024, 32768], seeds 0..255, theta from {0.3, 0.5, 0.7}, mixed precision,
    each run to t_end = 0.5, all admitted at once and advanced by the
    continuous-batching server (the clusters that reach their rebuild time
    in a launch are rebuilt together in one batched device build)."""
    import numpy as np
    import synth
    from paper_1602_02832_gb300 import serve

    members = synth.ensemble(a.ensemble, 1024, 32768, seed=0)
    t_end = a.ensemble_t_end
    reqs = []
    for k, mb in enumerate(members):
        x, v, m = synth.plummer(mb.n, mb.seed)
        reqs.append(serve.SimRequest(k, x, v, m, t_end))
    srvs = {}
    results, stats = [], None
    t0 = time.perf_counter()
    # one server per theta value (the opening angle is a per-context setting)
    tot = {"block_steps": 0, "interactions": 0, "step_us": [], "live": [], "launches": 0, "wall": 0.0,
           "phase_us": [0.0, 0.0]}
    for th in sorted({mb.theta for mb in members}):
        sub = [r for r, mb in zip(reqs, members) if mb.theta == th]
        srv = serve.Server(precision=hh.HH_MIXED, budget_bytes=150 * 10 ** 9, max_sims=256, max_steps=256,
                           theta=th, n_crit=a.n_crit, rebuild_threads=8,
                           rebuild_device=_server_rebuild(a),
                           order=hh.HH_ORDER_HILBERT if a.order == "hilbert" else hh.HH_ORDER_MORTON,
                           work_item=a.batch_work_item, work_split=a.batch_work_split)
        res, st = srv.run(sub, realtime=False)
        srv.close()
        results += res
        tot["block_steps"] += st.block_steps
        tot["interactions"] += st.interactions
        tot["step_us"] += st.step_us
        tot["live"] += st.live_per_step
        tot["launches"] += st.launches
        tot["wall"] += st.wall_s
        tot["phase_us"] = [u + w for u, w in zip(tot["phase_us"], st.phase_us)]
    wall = time.perf_counter() - t0
    lat = _lat(tot["step_us"])
    return {"clusters": len(members), "n_total": int(sum(mb.n for mb in members)), "t_end": t_end,
            "completed": len(results), "wall_s": wall, "launches": tot["launches"],
            "block_steps_per_s": tot["block_steps"] / wall, "interactions_per_s": tot["interactions"] / wall,
            "equiv_tflops": FLOP_PER_INT * tot["interactions"] / wall / 1e12,
            "mean_live_sims_per_step": float(np.mean(tot["live"])) if tot["live"] else None,
            "block_step_latency_us": lat,
            "device_s": {"predict_select": tot["phase_us"][0] * 1e-6, "force_correct": tot["phase_us"][1] * 1e-6},
            "note": "wall time includes admission (host tree build for the memory estimate, initial forces) "
                    "and the rebuilds; "
                    "block steps are summed over clusters; latency = device time of one global block step"}


def _lat_by_live(step_us, live):
    """Block-step latency (p50 / p99, microseconds) binned by the number of
    simulations in the launch that ran the step."""
    import numpy as np
    if not step_us:
        return None
    u, n = np.asarray(step_us), np.asarray(live)
    out = []
    lo = 1
    while lo <= n.max():
        hi = 2 * lo
        sel = (n >= lo) & (n < hi)
        if sel.any():
            out.append({"live": [int(lo), int(hi - 1)], "steps": int(sel.sum()),
                        "p50_us": float(np.quantile(u[sel], 0.5)), "p99_us": float(np.quantile(u[sel], 0.99))})
        lo = hi
    return out


def _queue_by_quarter(queue, wall_s):
    """Mean requests waiting (arrived, not yet resident) and mean resident
    simulations over each quarter of the window, from the per-launch samples:
    a queue that grows from quarter to quarter means the arrivals outrun the
    server."""
    out = []
    for q in range(4):
        lo, hi = wall_s * q / 4, wall_s * (q + 1) / 4
        s = [(w, r) for t, w, r in queue if lo <= t < hi]
        out.append({"quarter": q + 1, "launches": len(s),
                    "waiting_mean": sum(w for w, _ in s) / len(s) if s else None,
                    "resident_mean": sum(r for _, r in s) / len(s) if s else None})
    return out


def _lat_by_n(results, n_of):
    """Request latency (arrival to completion) by request size: N in
    [2^10, 2^12), [2^12, 2^14), [2^14, 2^16), [2^16, 2^18]."""
    import numpy as np

    out = []
    for lo in (1 << 10, 1 << 12, 1 << 14, 1 << 16):
        top = lo == 1 << 16
        u = [r.done_s - r.arrival_s for r in results
             if lo <= n_of[r.rid] and (n_of[r.rid] <= 4 * lo if top else n_of[r.rid] < 4 * lo)]
        if u:
            out.append({"n": [lo, 4 * lo if top else 4 * lo - 1], "completed": len(u),
                        "p50_s": float(np.quantile(u, 0.5)), "max_s": float(max(u))})
    return out or None


def _serving(hh, a, rate=20.0, seconds=None, launch_particles=0):
    """Serving: Poisson arrivals of Plummer + Salpeter cluster requests, N
    log-uniform in [2^10, 2^18], t_end in {1/8, 1/4, 1/2}, admitted within a
    150 GB device-memory budget, run for a bounded wall time.  With
    launch_particles, each launch advances at most that many particles."""
    import synth
    from paper_1602_02832_gb300 import serve

    seconds = a.serve_seconds if seconds is None else seconds
    n_req = max(1, int(rate * seconds))
    stream = synth.request_stream(n_req, rate_per_s=rate, seed=0)
    reqs = [serve.SimRequest(r.rid, None, None, None, r.t_end, arrival_s=r.arrival_s,
                             make=(lambda n=r.n, sd=r.seed: synth.plummer_salpeter(n, sd))) for r in stream]
    srv = serve.Server(precision=hh.HH_MIXED, budget_bytes=150 * 10 ** 9, max_sims=256, max_steps=32,
                       n_crit=a.n_crit, rebuild_threads=8, rebuild_device=_server_rebuild(a),
                       order=hh.HH_ORDER_HILBERT if a.order == "hilbert" else hh.HH_ORDER_MORTON,
                       launch_particles=launch_particles, work_item=a.batch_work_item,
                       work_split=a.batch_work_split)
    res, st = srv.run(reqs, realtime=True, max_wall_s=seconds)
    srv.close()
    arrived = sum(1 for r in stream if r.arrival_s <= st.wall_s)
    done_ids = {r.rid for r in res}
    # requests that arrived in the first half of the window: all of them
    # finish when the server keeps up with the arrivals (the longest request,
    # N = 2^18 to t = 1/2, takes several seconds under load)
    early = [r for r in stream if r.arrival_s <= st.wall_s / 2]
    return {"arrival_rate_per_s": rate, "window_s": seconds, "launch_particles": launch_particles or None,
            "requests_arrived": arrived, "completed": len(res),
            "completion_rate_per_s": len(res) / st.wall_s,
            "completed_of_first_half_arrivals": [sum(1 for r in early if r.rid in done_ids), len(early)],
            "unfinished_at_end": arrived - len(res),
            "queue_by_quarter": _queue_by_quarter(st.queue, st.wall_s),
            "wall_s": st.wall_s, "launches": st.launches,
            "block_steps_per_s": st.block_steps / st.wall_s, "interactions_per_s": st.interactions / st.wall_s,
            "block_step_latency_us": _lat(st.step_us),
            "block_step_latency_by_live": _lat_by_live(st.step_us, st.live_per_step),
            "request_latency_s": _lat([r.done_s - r.arrival_s for r in res],
                                      "wall seconds from a request's arrival to its completion") if res else None,
            "request_latency_by_n": _lat_by_n(res, {r.rid: r.n for r in stream}),
            "note": "requests arrive in real time over the window; unfinished ones are stopped at its end"}


def _j_from_tree(hh, x, v, m, T):
    """j arrays (particles in the tree's order, then its nodes), [nj, 3] / [nj]."""
    import numpy as np

    xj = np.concatenate([x[T.perm], T.node_x.T])
    vj = np.concatenate([v[T.perm], T.node_v.T])
    mj = np.concatenate([m[T.perm], T.node_m])
    return xj, vj, mj


def _config1(hh, a, peaks):
    """One force evaluation (acc, jerk, pot) of all N = 4096 particles of the
    seeded Plummer sphere (eps = 1e-4): by the direct sum (theta = 0: every
    list holds all particles, so every staged entry is shared by a whole i
    tile) and by the Barnes-Hut lists (theta = 0.5, leaf 8, n_crit 64); both
    precisions.  Device time of the force kernel (k_force) per evaluation,
    CUDA events on the context's stream, best of the repetitions."""
    import numpy as np
    import synth

    n, eps2 = 4096, 1e-8
    x, v, m = synth.plummer(n, 0)
    z = np.zeros((3, n))
    out = {"workload": "Plummer N=4096 (seed 0), eps=1e-4, one force evaluation of all particles; direct: "
                       "theta=0 lists (all N per group); tree: theta=0.5, leaf 8, n_crit 64",
           "note": "interactions = sum over particles of list length minus self; time = k_force device time "
                   "(CUDA events), best of the repetitions after two warm-up evaluations"}
    for lists, theta in (("direct", 0.0), ("tree", 0.5)):
        T = hh.hh_tree_build(x.T, v.T, z, z, m, leaf=8, n_crit=64, theta=theta)
        xj, vj, mj = _j_from_tree(hh, x, v, m, T)
        nj = len(mj)
        n_int = int((np.diff(T.off)[T.group_of] - 1).sum())
        for prec, name, peak_key in ((hh.HH_FP64, "fp64", "fp64_tflops"), (hh.HH_MIXED, "mixed", "fp32_tflops")):
            c = hh.hh_config_default()
            c.eps2, c.precision, c.theta, c.n_crit = eps2, prec, theta, 64
            c.tile_i = 32
            with hh.Context(c, n, nj, len(T.idx), T.n_groups) as ctx:
                ctx.hh_set_j(0, xj.T, vj.T, np.zeros((3, nj)), np.zeros((3, nj)), mj, np.zeros(nj))
                ctx.hh_set_lists(n, nj, T.off, T.idx, T.group_of)
                ctx.hh_predict(0.0)
                ia = np.arange(n, dtype=np.int32)
                for _ in range(2):
                    ctx.hh_force(ia, want=(False, False, False))
                best = math.inf
                for _ in range(5 if prec == hh.HH_FP64 else 30):
                    ctx.hh_force_timing(1)
                    ctx.hh_force(ia, want=(False, False, False))
                    ms, _ = ctx.hh_force_timing(0)
                    best = min(best, ms)
            ips = n_int / (best * 1e-3)
            tf = FLOP_PER_INT * ips / 1e12
            pk = peaks.get(peak_key)
            out[f"{lists}_{name}"] = {"interactions": n_int, "kernel_ms": best, "interactions_per_s": ips,
                                      "equiv_tflops": tf, "peak_tflops": pk, "frac": tf / pk if pk else None,
                                      "peak": f"measured {'FP64' if prec == hh.HH_FP64 else 'FP32'} FMA throughput "
                                              "(of measured)",
                                      "mean_list": float(np.diff(T.off).mean()), "groups": int(T.n_groups)}
    return out


def _config3(hh, torch, a, flush, peaks, over=None):
    """N = 2^20 Plummer sphere with a Salpeter mass spectrum (slope -2.35,
    mass ratio 100, total mass 1), mixed precision, 4th-order Hermite with
    block steps to t = 0.125 (eight 1/64 intervals, device rebuilds), theta
    0.5, leaf 8, eps 1e-4.  The whole run after set-up is timed (CUDA events
    on the context's stream).  Returns the figures and the data the CPU leg
    needs for its sampled oracle check."""
    import numpy as np
    import synth

    n = 1 << 20
    x, v, m = synth.plummer_salpeter(n, 0)
    cfg = _cfg(hh, hh.HH_MIXED, a)
    for k, val in (over or {}).items():
        setattr(cfg, k, val)
    ctx = hh.Context(cfg, n, 2 * n + 64, 16 * n + 4096, n // 4 + 64)
    stream = torch.cuda.Stream()
    ctx.hh_set_stream(stream.cuda_stream)
    w0 = time.perf_counter()
    ctx.hh_load_particles(x.T, v.T, m)
    ctx.hh_set_rebuild_device(True)
    ctx.hh_run(0.0, 0.0)
    setup_s = time.perf_counter() - w0
    loop = _Loop(hh, ctx, hh.HH_MIXED, "persistent")
    dtt = cfg.dt_tree
    t, t_end = 0.0, 0.125
    loop.enable(True)
    flush.zero_()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    while t < t_end:
        loop.advance(t + dtt)
        ctx.hh_rebuild(t + dtt)
        t += dtt
    e1.record(stream)
    e1.synchronize()
    loop.enable(False)
    ms = e0.elapsed_time(e1)
    c = ctx.hh_get_counters()
    hist = ctx.hh_get_tile_histogram().tolist()
    # sampled forces at t = 0.125 on the j entries and lists just rebuilt
    off, idx, gof = ctx.hh_get_lists()
    J = ctx.hh_get_j(0, ctx.nj)
    ctx.hh_predict(t_end)
    sample = np.sort(np.random.default_rng(3).choice(n, 200, replace=False)).astype(np.int32)
    gpu = ctx.hh_force(sample)
    dev_gb = ctx.device_bytes / 1e9
    loop.close()
    ctx.close()
    ips = c["interactions"] / (ms * 1e-3)
    force_ms = loop.phase_ms[1]
    tf_force = FLOP_PER_INT * c["interactions"] / (force_ms * 1e-3) / 1e12 if force_ms else None
    pk = peaks.get("fp32_tflops")
    res = {"workload": "Plummer N=2^20 with Salpeter masses (slope -2.35, ratio 100, M=1), seed 0, mixed precision, "
                       "4th-order Hermite block steps to t=0.125 (8 intervals of 1/64, device rebuilds), theta=0.5, "
                       f"leaf 8, n_crit {cfg.n_crit}, eps=1e-4",
           "value": ips, "unit": "interactions/s", "equiv_tflops": FLOP_PER_INT * ips / 1e12,
           "run_s": ms * 1e-3, "setup_s": setup_s, "device_gb": dev_gb,
           "block_steps_per_s": c["block_steps"] / (ms * 1e-3), "block_steps": c["block_steps"],
           "particle_steps": c["particle_steps"], "interactions": c["interactions"],
           "mean_list": c["interactions"] / max(1, c["particle_steps"]) + 1,
           "time_split_s": {"predict_select": loop.phase_ms[0] * 1e-3, "force": force_ms * 1e-3,
                            "rebuild_and_launch": ms * 1e-3 - (loop.phase_ms[0] + force_ms) * 1e-3},
           "block_step_latency_us": _lat(loop.step_us),
           "active_per_tile": _n_i({"n_i_hist": hist}),
           "roofline": {"kernel": "k_batch force phase (list force + corrector), mixed", "bound": "alu",
                        "achieved": tf_force, "peak": pk, "unit": "TFLOP/s",
                        "frac": tf_force / pk if (pk and tf_force) else None}}
    check = {"xj": np.ascontiguousarray(J["x"].T), "vj": np.ascontiguousarray(J["v"].T), "mj": J["m"],
             "off": off, "idx": idx, "gof": gof, "sample": sample, "gpu": gpu}
    return res, check


def _lat(vals, note="device time of one block step (all three phases) in the persistent loop"):
    import numpy as np
    if not vals:
        return None
    u = np.asarray(vals)
    return {"p50": float(np.quantile(u, 0.5)), "p99": float(np.quantile(u, 0.99)), "mean": float(u.mean()),
            "n": int(len(u)), "note": note}


def _n_i(r):
    """Active particles per evaluated i tile (the paper's n_i per staged list
    chunk): mean and histogram counts[k] for k + 1 active particles."""
    h = r.get("n_i_hist") or []
    tot = sum(h)
    if not tot:
        return None
    last = max(k for k, c in enumerate(h) if c)
    return {"mean": sum((k + 1) * c for k, c in enumerate(h)) / tot, "tiles": tot, "counts": h[:last + 1]}


def _split(r, steps):
    ph = r.get("phase_ms") or [0.0, 0.0, 0.0]
    if not any(ph):
        return {"force_kernel": r["force_ms"] / steps, "other": (r["ms"] - r["force_ms"]) / steps}
    return {"predict_select": ph[0] / steps, "force": ph[1] / steps, "correct": ph[2] / steps,
            "rebuild_and_launch": (r["ms"] - sum(ph)) / steps}


def _oracle_params(a):
    import oracle

    return oracle.RunParams(eps2=1e-8, eta=0.02, eta_s=0.01, dt_min=2.0 ** -30, dt_max=2.0 ** -6,
                            dt_tree=2.0 ** -6, theta=a.theta, leaf=8, n_crit=a.n_crit, use_tree=True)


def _cpu_baseline(a, state, cfg3=None):
    """The CPU leg: the FP64 oracle, as it stands, on the host cores.
    (1) Timed on a bounded sample of the timed window: resumed from the GPU
    arm's synchronised state at the start of its first timed interval, over
    its first four intervals, rebuilds included (the same block steps, lists
    and interactions, up to rounding).  (2) With cfg3, the oracle's list force on
    the sampled particles of the N = 2^20 run, on the GPU's own j entries and
    lists, compared with the GPU's forces."""
    import numpy as np
    import oracle

    oracle.build()
    p = _oracle_params(a)
    t0 = state["t"]
    w0 = time.perf_counter()
    t1 = t0 + min(CPU_BASELINE_T, a.steps * p.dt_tree)
    r = oracle.resume(state["x"], state["v"], state["a"], state["jk"], state["dt"], state["m"], t0, t1, p)
    dt = time.perf_counter() - w0
    out = {"value": r["stats"]["interactions"] / dt, "unit": "interactions/s", "cores": oracle.num_threads(),
           "kind": "oracle",
           "sample": f"FP64 oracle tree loop resumed from the GPU arm's state at t = {t0:g} (the start of its "
                     f"first timed interval, N={a.n}) over t in [{t0:g}, {t1:g}] "
                     f"({r['stats']['particle_steps']} particle steps, {r['stats']['interactions']} "
                     f"interactions, {dt:.1f} s)"}
    if cfg3:
        s = cfg3["sample"]
        w0 = time.perf_counter()
        ra, rj, rp = oracle.list_force(cfg3["xj"], cfg3["vj"], cfg3["mj"], s, cfg3["gof"][s], cfg3["off"],
                                       cfg3["idx"], 1e-8)
        dt3 = time.perf_counter() - w0
        acc, jerk, pot = cfg3["gpu"]
        ea = np.linalg.norm(acc.T - ra, axis=1) / np.linalg.norm(ra, axis=1)
        ej = np.linalg.norm(jerk.T - rj, axis=1) / np.linalg.norm(rj, axis=1)
        ep = np.abs(pot - rp) / np.abs(rp)
        n_int = int((np.diff(cfg3["off"])[cfg3["gof"][s]] - 1).sum())
        out["config3_check"] = {
            "particles": int(len(s)), "acc_max_rel": float(ea.max()), "jerk_max_rel": float(ej.max()),
            "jerk_p999_rel": float(np.quantile(ej, 0.999)), "pot_max_rel": float(ep.max()),
            "bars": "acc, pot <= 1e-6; jerk <= 1e-5 (or <= 1e-6 of J_scale where it nearly cancels)",
            "oracle_interactions_per_s": n_int / dt3,
            "note": "mixed-form forces of sampled particles at t = 0.125 against the FP64 oracle's list force "
                    "on the same j entries and lists"}
    return out


def main_reference(a):
    """The FP64 oracle as the reference arm, on the host cores: the same
    workload run from t = 0 to the start of the GPU arm's timed window (W
    intervals of 1/64), then each step is the oracle resumed from that
    synchronised state over the first quarter of the next interval."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    import synth

    oracle.build()
    x, v, m = synth.plummer(a.n, 0)
    p = _oracle_params(a)
    t0 = a.warmup * p.dt_tree
    w0 = time.perf_counter()
    r0 = oracle.run(x, v, m, t0, p)
    prep_s = time.perf_counter() - w0
    st = (r0["x"], r0["v"], r0["a"], r0["jk"], r0["dt"], m, t0, t0 + CPU_SAMPLE_T, p)
    for _ in range(a.warmup):
        oracle.resume(*st)
    tot_int, tot_s, tot_bs = 0, 0.0, 0
    for _ in range(a.steps):
        w0 = time.perf_counter()
        r = oracle.resume(*st)
        tot_s += time.perf_counter() - w0
        tot_int += r["stats"]["interactions"]
        tot_bs += r["stats"]["block_steps"]
    val = tot_int / tot_s
    sample = (f"each step: FP64 oracle tree loop of N={a.n} Plummer resumed from its own state at t = {t0:g} "
              f"(reached by an untimed run from t = 0 in {prep_s:.1f} s: the start of the GPU arm's timed window) "
              f"over t in [{t0:g}, {t0 + CPU_SAMPLE_T:g}]")
    # n_gpus is the launch's N (the oracle itself runs on rank 0's host cores)
    line = {"metric": METRIC, "value": val, "unit": "interactions/s", "n_gpus": max(world, a.gpus), "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": tot_s * 1e3 / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": _workload(a), "n": a.n, "form": "oracle fp64 (CPU)"},
            "equiv_tflops": FLOP_PER_INT * val / 1e12,
            "block_steps_per_s": tot_bs / tot_s,
            "cpu_baseline": {"value": val, "unit": "interactions/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    a = _args()
    if a.impl == "reference":
        return main_reference(a)
    world, rank, local = _dist()
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build_library()
    if world > 1:
        dist.barrier()
    import paper_1602_02832_gb300 as hh

    peaks = _peaks(os.path.dirname(hh.LIB_PATH), local) if rank == 0 else {}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    if a.mixed_only:
        r = _run_form(hh, torch, a, hh.HH_MIXED, rank, a.steps, a.warmup, flush)
        if rank == 0:
            print(json.dumps({"form": "mixed", "value": r["interactions"] / (r["ms"] * 1e-3), "ms": r["ms"],
                              "force_ms": r["force_ms"]}), flush=True)
        return 0
    best64, table64 = _tuned(hh, a, hh.HH_FP64, rank)
    bestmx, tablemx = _tuned(hh, a, hh.HH_MIXED, rank) if not a.no_mixed else ({}, None)
    with Clocks(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        res = _run_form(hh, torch, a, hh.HH_FP64, rank, a.steps, a.warmup, flush, e2e_steps=a.steps, over=best64,
                        keep_state=True)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    mixed = None
    if not a.no_mixed:
        mixed = _run_form(hh, torch, a, hh.HH_MIXED, rank, a.steps, a.warmup, flush, over=bestmx)
    cfg3, cfg3_check = (None, None)
    if not a.no_config3 and rank == 0:
        cfg3, cfg3_check = _config3(hh, torch, a, flush, peaks, over=bestmx)
    cfg1 = _config1(hh, a, peaks) if (not a.no_config1 and rank == 0) else None
    tot, mx = reduce_over_ranks(
        [res["interactions"], res["block_steps"], res["particle_steps"], res["gpu_launches"], res["e2e"]["interactions"]],
        [res["ms"], res["e2e"]["ms"]], torch.device("cuda", local), world)
    if rank == 0:
        value = tot[0] / (mx[0] * 1e-3)
        achieved = FLOP_PER_INT * res["interactions"] / (res["force_ms"] * 1e-3) / 1e12
        cpu = None if (a.no_cpu_baseline or world > 1) else _cpu_baseline(a, res["warm_state"], cfg3_check)
        line = {
            "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": mx[0] / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Plummer spheres, seed = rank)",
            "config": {"workload": _workload(a), "n": a.n, "theta": a.theta,
                       "n_crit": best64.get("n_crit", a.n_crit),
                       "form": "plain FP64", "replicas": world,
                       "l2": "flushed (256 MB write) before every timed step"},
            "equiv_tflops": FLOP_PER_INT * value / 1e12,
            "equiv_tflops_57": 57 * value / 1e12,
            "block_steps_per_s": tot[1] / (mx[0] * 1e-3),
            "particle_steps_per_s": tot[2] / (mx[0] * 1e-3),
            "roofline": {"kernel": ("k_batch force phase (list force + corrector), plain FP64"
                                    if a.loop == "persistent"
                                    else "k_force<RecF64> (plain FP64 list force)"),
                         "bound": "alu",
                         "achieved": achieved, "peak": peaks.get("fp64_tflops"), "unit": "TFLOP/s",
                         "frac": achieved / peaks["fp64_tflops"] if peaks.get("fp64_tflops") else None,
                         "traffic": _traffic(res["shape"]) if a.loop == "persistent" else None,
                         "traffic_capture": TRAFFIC_FP64["capture"],
                         "note": "achieved = 60 algorithmic flop per interaction / device time of the force "
                                 "phases (persistent loop: %globaltimer stamps at the phase barriers, the phase "
                                 "includes the corrector of each completed tile; graph loop: CUDA events around "
                                 "the force kernel); peak = measured FP64 FMA throughput "
                                 "(of measured, libhh_peaks.so); traffic = DRAM bytes of one k_batch launch "
                                 "(one interval, all phases) from one ncu capture of that launch "
                                 "(traffic_capture), null when the kernel sources or the tile shape differ from the "
                                 "captured ones"},
            "e2e": {"value": tot[4] / (mx[1] * 1e-3), "unit": "interactions/s",
                    "h2d_bytes_per_step": res["e2e"]["bi"], "d2h_bytes_per_step": res["e2e"]["bo"]},
            "gpu_launches": int(tot[3]),
            "loop": a.loop,
            "rebuild": a.rebuild,
            "order": a.order,
            "tuning": {"fp64": {"chosen": best64, "candidates": table64},
                       "mixed": {"chosen": bestmx, "candidates": tablemx},
                       "note": "autotuner runs before the timed region (paper_1602_02832_gb300/autotune.py)"},
            "time_split_ms_per_step": _split(res, a.steps),
            "block_step_latency_us": _lat(res["step_us"]),
            "active_per_tile": _n_i(res),
            "force_kernel_share": res["force_ms"] / res["ms"],
            "peaks_measured": peaks,
        }
        if mixed:
            mv = mixed["interactions"] / (mixed["ms"] * 1e-3)
            mach = FLOP_PER_INT * mixed["interactions"] / (mixed["force_ms"] * 1e-3) / 1e12
            line["mixed"] = {
                "value": mv, "unit": "interactions/s", "equiv_tflops": FLOP_PER_INT * mv / 1e12,
                "block_steps_per_s": mixed["block_steps"] / (mixed["ms"] * 1e-3),
                "ms_per_step": mixed["ms"] / a.steps, "force_kernel_share": mixed["force_ms"] / mixed["ms"],
                "speedup_vs_plain": mv / (res["interactions"] / (res["ms"] * 1e-3)),
                "time_split_ms_per_step": _split(mixed, a.steps),
                "block_step_latency_us": _lat(mixed["step_us"]),
                "active_per_tile": _n_i(mixed),
                "roofline": {"kernel": ("k_batch force phase (list force + corrector), mixed"
                                        if a.loop == "persistent" else "k_force<RecMix> (mixed list force)"),
                             "bound": "alu", "achieved": mach,
                             "peak": peaks.get("fp32_tflops"), "unit": "TFLOP/s",
                             "frac": mach / peaks["fp32_tflops"] if peaks.get("fp32_tflops") else None},
            }
        if cfg3:
            line["config3"] = cfg3
        if cfg1:
            line["config1"] = cfg1
        if a.ensemble > 0:
            line["batched"] = _ensemble(hh, a)
            line["batched"]["block_steps_per_s_vs_plain"] = line["batched"]["block_steps_per_s"] / line["block_steps_per_s"]
        if a.serve_seconds > 0:
            line["serving"] = _serving(hh, a, launch_particles=a.serve_launch_particles)
            if a.serve_sustained_rate > 0:
                line["serving_sustained"] = _serving(hh, a, rate=a.serve_sustained_rate,
                                                     seconds=a.serve_sustained_seconds,
                                                     launch_particles=a.serve_launch_particles)
        line["clocks"] = clk.summary()
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
