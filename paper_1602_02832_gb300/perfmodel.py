"""GPU analogue of the paper's breakdown of the calculation time (Section 3,
Table 1) and a fit of its force-time model (Eq. 3).

The paper splits the time per particle step into T_grape (force and jerk on
GRAPE-9), T_tree (tree and lists on the host, step 1), T_comm (host <->
GRAPE transfers) and T_host (the rest of the host's integration), and models
T_grape = N_int t_pipe (n_i / n_pipe)^-1, where N_int is the mean list length
and n_i the mean number of particles that are evaluated together (one group's
active particles in a block step).

Here, with the tree loop running on the GPU (`hh_batch_run`, device rebuilds):
- T_force: the force phase of each block step (list force and, for each tile
  whose forces are complete, the corrector), device time;
- T_predict: the predict + select phase, device time;
- T_tree: the device rebuild every dt_tree, wall time of hh_rebuild;
- T_host: wall time of the loop minus the device phases (launch and host
  bookkeeping);
- T_comm: the loop moves no particle data between host and GPU per step; the
  column gives, for context, a full state round trip (hh_get_state + hh_set_j)
  per tree interval spread over that interval's particle steps.
N_int = interactions / particle steps.  n_i = particle steps / active tile
steps: the particles that share one staged list chunk (at most tile_i).

The force-time model T_force / N_int = t_int + t_stage / n_i (t_int: time
per interaction when staging is fully shared; t_stage: time to stage one
list entry for a tile; t_stage / t_int plays the role of the paper's n_pipe,
the n_i below which sharing, not arithmetic, sets the rate) is fitted on a
controlled sweep: one force evaluation (hh_force, the same list-force body)
on active sets with exactly k active particles in every i tile, k = 1 ... 32,
timed with CUDA events around the force kernel.  The tree-loop runs give
n_i of only ~4-6, too narrow a range to separate the two terms.

Usage (on a GPU): python -m paper_1602_02832_gb300.perfmodel --out DIR
List run statistics (host only): python -m paper_1602_02832_gb300.perfmodel --list-runs
Per-step profile of one tree interval (on a GPU):
    python -m paper_1602_02832_gb300.perfmodel --step-profile --n 65536 --form fp64 \
        --cfg '{"n_crit": 64, "tile_i": 8, "tile_j": 256, "work_item": 2048, "work_split": 2048, "tile_j_small": 64}'
T_tree of many simulations, one by one against one batched build (on a GPU):
    python -m paper_1602_02832_gb300.perfmodel --rebuild-batch 85            # N log-uniform in [1024, 32768]
    python -m paper_1602_02832_gb300.perfmodel --rebuild-batch 64 --n 1024   # 64 of one size
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

# The paper's Table 1 (GRAPE-9, n_crit = 4000, dt_tree = 1/64): N, theta,
# N_int, n_i, T_grape, T_tree, T_comm, T_host (seconds per particle step).
PAPER_TABLE1 = [
    (65536, 0.75, 5740, 29.3, 8.5e-6, 1.5e-7, 9.8e-7, 1.6e-7),
    (65536, 0.5, 11081, 28.8, 1.6e-5, 2.4e-7, 9.8e-7, 1.6e-7),
    (65536, 0.3, 22351, 28.6, 3.3e-5, 4.0e-7, 9.8e-7, 1.5e-7),
    (262144, 0.75, 6433, 29.8, 9.2e-6, 9.7e-8, 1.2e-6, 2.7e-7),
    (262144, 0.5, 12644, 29.5, 1.8e-5, 1.5e-7, 1.2e-6, 2.7e-7),
    (262144, 0.3, 28168, 29.4, 4.0e-5, 2.7e-7, 1.2e-6, 2.6e-7),
]


def measure(n, theta, n_crit, precision, intervals=2, warm=1, seed=0, tile_i=0, tile_j=0):
    """Runs the tree loop of a seeded Plummer sphere (standard units, eps^2 =
    1e-8, eta = 0.02, dt_tree = 1/64) for `warm` + `intervals` tree intervals
    from t = 0 and returns the per-particle-step breakdown of the timed ones."""
    import synth
    from . import HH_FP64, Batch, Context, hh_config_default, hh_tree_build

    x, v, m = synth.plummer(n, seed)
    cfg = hh_config_default()
    cfg.eps2, cfg.eta, cfg.theta, cfg.n_crit, cfg.precision = 1e-8, 0.02, theta, n_crit, precision
    cfg.tile_i, cfg.tile_j = tile_i, tile_j
    z = np.zeros((3, n))
    T = hh_tree_build(x.T, v.T, z, z, m, leaf=cfg.leaf, n_crit=n_crit, theta=theta)
    dtt = cfg.dt_tree
    with Context(cfg, n, 2 * n, 2 * len(T.idx) + 4096, 2 * T.n_groups + 64) as ctx, \
            Batch(precision, max_sims=1, max_steps=4096) as b:
        ctx.hh_load_particles(np.ascontiguousarray(x.T), np.ascontiguousarray(v.T), m)
        ctx.hh_set_rebuild_device(True)
        ctx.hh_run(0.0, 0.0)
        t = 0.0
        acc = dict(wall=0.0, phase=np.zeros(3), rebuild=0.0, comm=0.0)
        c0 = None
        for k in range(warm + intervals):
            timed = k >= warm
            if timed and c0 is None:
                c0 = ctx.hh_get_counters()
            w = time.perf_counter()
            while True:
                _, tn, _ = b.hh_batch_run([ctx], [t + dtt])
                if timed:
                    acc["phase"] += b.last_phase_us.sum(0) * 1e-6
                if tn[0] > t + dtt:
                    break
            if timed:
                acc["wall"] += time.perf_counter() - w
            w = time.perf_counter()
            ctx.hh_rebuild(t + dtt)
            if timed:
                acc["rebuild"] += time.perf_counter() - w
            t += dtt
            if timed:  # context for T_comm: one state round trip per interval
                w = time.perf_counter()
                st = ctx.hh_get_state()
                ids = ctx.hh_get_ids()
                ctx.hh_set_j(0, st["x"], st["v"], st["a"], st["jk"], np.ascontiguousarray(m[ids]), st["t"])
                acc["comm"] += time.perf_counter() - w
        c1 = ctx.hh_get_counters()
    ps = c1["particle_steps"] - c0["particle_steps"]
    n_int = (c1["interactions"] - c0["interactions"]) / ps
    n_i = ps / max(1, c1["tile_steps"] - c0["tile_steps"])
    ph = acc["phase"]
    return {
        "n": n, "theta": theta, "n_crit": n_crit, "form": "fp64" if precision == HH_FP64 else "mixed",
        "particle_steps": int(ps), "block_steps": int(c1["block_steps"] - c0["block_steps"]),
        "N_int": n_int, "n_i": n_i,
        "T_force": ph[1] / ps, "T_predict": ph[0] / ps, "T_tree": acc["rebuild"] / ps,
        "T_host": max(0.0, acc["wall"] - ph.sum()) / ps, "T_comm_round_trip": acc["comm"] / ps,
    }


def equivalent_performance(n, precision, theta=0.5, n_crit=64, intervals=1, warm=1, seed=0):
    """The paper's equivalent performance S = 57 N n_step,h / T (Eq. 1): the
    speed a direct Hermite code would need to reach the tree code's time to
    solution.  n_step,h comes from the same loop with theta = 0 (every list is
    all particles, i.e. direct Hermite with the same block steps), over the
    same tree intervals as the tree run timed for T.  Returns S for the tree
    run and the tree and direct runs' rates."""
    tree = measure(n, theta, n_crit, precision, intervals, warm, seed)
    direct = measure(n, 0.0, n_crit, precision, intervals, warm, seed)
    t_tree = tree["particle_steps"] * (tree["T_force"] + tree["T_predict"] + tree["T_tree"] + tree["T_host"])
    t_direct = direct["particle_steps"] * (direct["T_force"] + direct["T_predict"] + direct["T_tree"] +
                                           direct["T_host"])
    return {"n": n, "form": tree["form"], "theta": theta, "n_crit": n_crit, "intervals": intervals,
            "steps_ratio_direct_over_tree": direct["particle_steps"] / tree["particle_steps"],
            "S_tree_tflops": 57.0 * direct["particle_steps"] * n / t_tree / 1e12,
            "tree_interactions_per_s": tree["N_int"] * tree["particle_steps"] / t_tree,
            "direct_interactions_per_s": direct["N_int"] * direct["particle_steps"] / t_direct,
            "speedup_over_direct": t_direct / t_tree}


def _tiles(off, group_of, tile_i):
    """Static i tiles (begin, end) as the library forms them: runs of at most
    tile_i consecutive particles inside each group (groups are contiguous in
    Morton order)."""
    g = np.asarray(group_of)
    starts = np.r_[0, np.nonzero(np.diff(g))[0] + 1]
    ends = np.r_[starts[1:], len(g)]
    out = []
    for b, e in zip(starts, ends):
        for q in range(b, e, tile_i):
            out.append((q, min(q + tile_i, e)))
    return out


def sweep_n_i(n, theta, n_crit, precision, ks=(1, 2, 4, 8, 16, 32), reps=5, seed=0, tile_i=32):
    """Force time per interaction against the number k of active particles
    per i tile (the paper's n_i), from hh_force on a tree at t = 0."""
    import synth
    from . import HH_FP64, Context, hh_config_default, hh_tree_build

    x, v, m = synth.plummer(n, seed)
    cfg = hh_config_default()
    cfg.eps2, cfg.theta, cfg.n_crit, cfg.precision, cfg.tile_i = 1e-8, theta, n_crit, precision, tile_i
    z = np.zeros((3, n))
    T = hh_tree_build(x.T, v.T, z, z, m, leaf=cfg.leaf, n_crit=n_crit, theta=theta)
    rows = []
    with Context(cfg, n, 2 * n, 2 * len(T.idx) + 4096, 2 * T.n_groups + 64) as ctx:
        ctx.hh_load_particles(np.ascontiguousarray(x.T), np.ascontiguousarray(v.T), m)
        ctx.hh_set_rebuild_device(True)
        ctx.hh_run(0.0, 0.0)
        off, idx, gof = ctx.hh_get_lists()
        length = np.diff(off)[gof] - 1  # interactions of each particle (self excluded)
        tiles = _tiles(off, gof, tile_i)
        ctx.hh_predict(0.0)
        for k in ks:
            act = np.concatenate([np.arange(b, min(b + k, e)) for b, e in tiles]).astype(np.int32)
            ctx.hh_force(act, want=(False, False, False))  # warm-up
            best = math.inf
            for _ in range(reps):
                ctx.hh_force_timing(1)
                ctx.hh_force(act, want=(False, False, False))
                ms, _ = ctx.hh_force_timing(0)
                best = min(best, ms * 1e-3)
            n_int = float(length[act].sum())
            rows.append({"form": "fp64" if precision == HH_FP64 else "mixed", "n": n, "theta": theta,
                         "n_crit": n_crit, "k": k, "n_act": int(len(act)), "n_i": float(len(act)) / len(tiles),
                         "N_int": n_int / len(act), "T_force": best / len(act), "time_s": best,
                         "interactions_per_s": n_int / best})
    return rows


def fit_force_model(rows):
    """Least-squares fit of T_force / N_int = t_int + t_stage / n_i over rows
    of one form.  Returns t_int, t_stage, n_pipe = t_stage / t_int and the
    coefficient of determination of the fit."""
    y = np.array([r["T_force"] / r["N_int"] for r in rows], dtype=np.float64)
    x = np.array([1.0 / r["n_i"] for r in rows], dtype=np.float64)
    A = np.stack([np.ones_like(x), x], axis=1)
    (t_int, t_stage), *_ = np.linalg.lstsq(A, y, rcond=None)
    pred = A @ np.array([t_int, t_stage])
    ss_res = float(((y - pred) ** 2).sum())
    ss_tot = float(((y - y.mean()) ** 2).sum())
    return {"t_int": float(t_int), "t_stage": float(t_stage),
            "n_pipe": float(t_stage / t_int) if t_int > 0 else math.inf,
            "r2": 1.0 - ss_res / ss_tot if ss_tot > 0 else 1.0, "points": len(rows)}


def sweep_markdown(rows, fits):
    lines = ["| form | N | theta | n_crit | k active per tile | n_i | N_int | force time (s) | T_force / N_int (s) | "
             "interactions/s |", "|---|---:|---:|---:|---:|---:|---:|---:|---:|---:|"]
    for r in rows:
        lines.append(f"| {r['form']} | {r['n']} | {r['theta']} | {r['n_crit']} | {r['k']} | {r['n_i']:.2f} | "
                     f"{r['N_int']:.0f} | {r['time_s']:.3e} | {r['T_force'] / r['N_int']:.3e} | "
                     f"{r['interactions_per_s']:.3e} |")
    lines += ["", "Fit T_force / N_int = t_int + t_stage / n_i over the sweep:", "",
              "| form | t_int (s) | t_stage (s) | n_pipe = t_stage / t_int | R^2 | points |",
              "|---|---:|---:|---:|---:|---:|"]
    for form, f in fits.items():
        lines.append(f"| {form} | {f['t_int']:.3e} | {f['t_stage']:.3e} | {f['n_pipe']:.1f} | {f['r2']:.3f} | "
                     f"{f['points']} |")
    return "\n".join(lines) + "\n"


def table_markdown(rows, fits):
    lines = ["| form | N | theta | n_crit | N_int | n_i | T_force | T_predict | T_tree | T_host | "
             "T_comm (round trip) |", "|---|---:|---:|---:|---:|---:|---:|---:|---:|---:|---:|"]
    for r in rows:
        lines.append(f"| {r['form']} | {r['n']} | {r['theta']} | {r['n_crit']} | {r['N_int']:.0f} | {r['n_i']:.1f} | "
                     f"{r['T_force']:.2e} | {r['T_predict']:.2e} | {r['T_tree']:.2e} | {r['T_host']:.2e} | "
                     f"{r['T_comm_round_trip']:.2e} |")
    if fits:
        lines += ["", "Fit T_force / N_int = t_int + t_stage / n_i over these runs:", "",
                  "| form | t_int (s) | t_stage (s) | n_pipe = t_stage / t_int | R^2 | points |",
                  "|---|---:|---:|---:|---:|---:|"]
        for form, f in fits.items():
            lines.append(f"| {form} | {f['t_int']:.3e} | {f['t_stage']:.3e} | {f['n_pipe']:.1f} | {f['r2']:.3f} | "
                         f"{f['points']} |")
    lines += ["", "Paper, Table 1 (GRAPE-9, n_crit 4000; seconds per particle step):", "",
              "| N | theta | N_int | n_i | T_grape | T_tree | T_comm | T_host |", "|---:|---:|---:|---:|---:|---:|---:|---:|"]
    for row in PAPER_TABLE1:
        lines.append("| " + " | ".join(str(u) for u in row) + " |")
    return "\n".join(lines) + "\n"


def list_run_stats(off, idx, n_particles, rec_bytes=(48, 64)):
    """Run statistics of CSR interaction lists, for the (start, count) encoding
    of the paper's cell-index memory (Section 2): a run is a maximal stretch
    of one list whose entries are consecutive j indices.  Returns entries,
    runs and entries per run (all, particle entries < n_particles, node
    entries), index bytes as 4-byte CSR entries and as 8-byte (start, count)
    pairs, and the share of index bytes in the staged bytes of each record
    size (record + its 4-byte index)."""
    off = np.asarray(off, dtype=np.int64)
    idx = np.asarray(idx, dtype=np.int64)
    L = int(off[-1])
    idx = idx[:L]
    starts = np.ones(L, dtype=bool)
    if L > 1:
        starts[1:] = idx[1:] != idx[:-1] + 1
    first = off[:-1][off[1:] > off[:-1]]  # a run never crosses into the next list
    starts[first] = True
    is_p = idx < n_particles
    out = {"entries": L, "runs": int(starts.sum()),
           "entries_per_run": L / max(1, int(starts.sum())),
           "particle_entries_per_run": int(is_p.sum()) / max(1, int((starts & is_p).sum())),
           "node_entries_per_run": int((~is_p).sum()) / max(1, int((starts & ~is_p).sum())),
           "index_bytes_csr": 4 * L, "index_bytes_ranges": 8 * int(starts.sum())}
    out["range_bytes_over_csr"] = out["index_bytes_ranges"] / max(1, out["index_bytes_csr"])
    for rb in rec_bytes:
        out[f"index_share_of_staged_{rb}B"] = 4.0 / (rb + 4.0)
    return out


def list_runs_main(argv=None):
    """Run statistics of the library's host-built lists for Plummer spheres
    (no GPU needed): python -m paper_1602_02832_gb300.perfmodel --list-runs"""
    import synth
    from . import HH_ORDER_HILBERT, HH_ORDER_MORTON, hh_tree_build

    p = argparse.ArgumentParser()
    p.add_argument("--list-runs", action="store_true")
    p.add_argument("--n", type=int, nargs="+", default=[65536])
    p.add_argument("--theta", type=float, nargs="+", default=[0.5])
    p.add_argument("--n-crit", type=int, nargs="+", default=[64, 4000])
    a = p.parse_args(argv)
    rows = []
    for n in a.n:
        x, v, m = synth.plummer(n, 0)
        z = np.zeros((3, n))
        for th in a.theta:
            for nc in a.n_crit:
                for order, name in ((HH_ORDER_MORTON, "morton"), (HH_ORDER_HILBERT, "hilbert")):
                    T = hh_tree_build(x.T, v.T, z, z, m, leaf=8, n_crit=nc, theta=th, order=order)
                    r = dict(n=n, theta=th, n_crit=nc, order=name, **list_run_stats(T.off, T.idx, n))
                    rows.append(r)
                    print(json.dumps(r), flush=True)
    return rows


STEP_EDGES = (1, 9, 33, 129, 513, 2049, 8193, 32769, 131073, 1 << 40)


def step_profile(n, precision, cfg=None, salpeter=False, warm=2, seed=0):
    """One tree interval of the batched loop (`hh_batch_run`, device
    rebuilds), step by step: the seeded Plummer sphere (with Salpeter masses
    if `salpeter`) is advanced `warm` intervals, then the next interval runs
    twice from the same state, once in one launch (each block step's device
    phase times from the kernel's stamps) and once one block step per launch
    (each step's active particles, interactions and list mode from the
    counters).  Both runs take the same steps.  Returns an array of rows
    (active particles, interactions, list mode, step us, select + predict
    us, force + correct us)."""
    import synth
    from . import Batch, Context, hh_config_default, hh_tree_build

    def make():
        x, v, m = (synth.plummer_salpeter if salpeter else synth.plummer)(n, seed)
        c = hh_config_default()
        c.eps2, c.eta, c.theta, c.precision = 1e-8, 0.02, 0.5, precision
        for k, val in (cfg or {}).items():
            setattr(c, k, val)
        z = np.zeros((3, n))
        T0 = hh_tree_build(x.T, v.T, z, z, m, leaf=8, n_crit=c.n_crit, theta=c.theta)
        ctx = Context(c, n, 2 * n, 2 * len(T0.idx) + 1024, 2 * T0.n_groups + 64)
        ctx.hh_load_particles(x.T, v.T, m)
        ctx.hh_set_rebuild_device(True)
        ctx.hh_run(0.0, 0.0)
        return ctx, c.dt_tree

    def interval(b, ctx, t, dtt):
        us, ph = [], []
        while True:
            steps, tn, u = b.hh_batch_run([ctx], [t + dtt])
            if steps:
                us.append(np.array(u[:steps]))
                ph.append(np.array(b.last_phase_us[:steps]))
            if tn[0] > t + dtt:
                return np.concatenate(us), np.concatenate(ph)

    ca, dtt = make()
    cb, _ = make()
    with ca, cb, Batch(precision, max_sims=1, max_steps=8192) as b:
        t = 0.0
        for _ in range(warm):
            for ctx in (ca, cb):
                interval(b, ctx, t, dtt)
                ctx.hh_rebuild(t + dtt)
            t += dtt
        U, PH = interval(b, cb, t, dtt)
        rows = []
        while True:
            c0 = ca.hh_get_counters()
            steps, tn, _ = b.hh_batch_run([ca], [t + dtt], max_steps=1)
            c1 = ca.hh_get_counters()
            if steps:
                rows.append((c1["particle_steps"] - c0["particle_steps"], c1["interactions"] - c0["interactions"],
                             c1["list_steps"] - c0["list_steps"]))
            if tn[0] > t + dtt:
                break
    if len(rows) != len(U):
        raise RuntimeError(f"the two runs took {len(rows)} and {len(U)} steps")
    r = np.array(rows, dtype=np.float64)
    return np.column_stack([r, U, PH[:, 0], PH[:, 1] + PH[:, 2]])


def step_bins(rows, edges=STEP_EDGES):
    """Per-step rows (step_profile) binned by active particles [lo, hi):
    steps, list-mode steps, time and interaction shares, sums and medians of
    the two phases, and the force phase's interaction rate."""
    rows = np.asarray(rows, dtype=np.float64)
    A, I, LM, U, P1, P2 = rows.T
    out = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        s = (A >= lo) & (A < hi)
        if not s.any():
            continue
        out.append({"active": [int(lo), int(hi - 1)], "steps": int(s.sum()), "list_steps": int(LM[s].sum()),
                    "time_share": float(U[s].sum() / U.sum()), "interaction_share": float(I[s].sum() / I.sum()),
                    "select_predict_us_sum": float(P1[s].sum()), "select_predict_us_median": float(np.median(P1[s])),
                    "force_us_sum": float(P2[s].sum()), "force_us_median": float(np.median(P2[s])),
                    "force_rate": float(I[s].sum() / (P2[s].sum() * 1e-6)) if P2[s].sum() > 0 else None})
    return out


def step_profile_main(argv=None):
    from . import HH_FP64, HH_MIXED

    p = argparse.ArgumentParser()
    p.add_argument("--step-profile", action="store_true")
    p.add_argument("--n", type=int, default=65536)
    p.add_argument("--form", default="fp64", choices=["fp64", "mixed"])
    p.add_argument("--salpeter", action="store_true")
    p.add_argument("--warm", type=int, default=2)
    p.add_argument("--cfg", default="{}", help="hh_config fields as JSON")
    a = p.parse_args(argv)
    rows = step_profile(a.n, HH_FP64 if a.form == "fp64" else HH_MIXED, json.loads(a.cfg), a.salpeter, a.warm)
    A, I, LM, U, P1, P2 = rows.T
    print(json.dumps({"n": a.n, "form": a.form, "salpeter": a.salpeter, "steps": len(rows),
                      "interval_ms": float(U.sum() / 1e3), "select_predict_ms": float(P1.sum() / 1e3),
                      "force_ms": float(P2.sum() / 1e3), "interactions": float(I.sum()),
                      "list_steps": int(LM.sum())}), flush=True)
    for b in step_bins(rows):
        print(json.dumps(b), flush=True)
    return rows


def rebuild_batch(ns, precision, reps=5, warm=2, seed=0):
    """T_tree of many simulations: wall time of rebuilding K contexts (Plummer
    spheres of sizes ns, seeds seed + k, device builders) one after another
    with hh_rebuild and together with one hh_batch_rebuild, each averaged
    over reps after warm rounds of both."""
    import numpy as np
    import synth
    from . import Batch, Context, hh_config_default
    ctxs = []
    try:
        for k, n in enumerate(ns):
            x, v, m = synth.plummer(int(n), seed + k)
            c = hh_config_default()
            c.eps2, c.precision, c.n_crit = 1e-8, precision, 64
            ctx = Context(c, int(n), 2 * int(n) + 64, 400 * int(n) + 4096, int(n) + 64)
            ctxs.append(ctx)
            ctx.hh_load_particles(x.T, v.T, m)
            ctx.hh_set_rebuild_device(True)
        with Batch(precision, max_sims=max(1, len(ns)), max_steps=8) as b:
            for _ in range(warm):
                for ctx in ctxs:
                    ctx.hh_rebuild(0.0)
                b.hh_batch_rebuild(ctxs, 0.0)
            t0 = time.perf_counter()
            for _ in range(reps):
                for ctx in ctxs:
                    ctx.hh_rebuild(0.0)
            t1 = time.perf_counter()
            for _ in range(reps):
                b.hh_batch_rebuild(ctxs, 0.0)
            t2 = time.perf_counter()
    finally:
        for ctx in ctxs:
            ctx.close()
    one, many = (t1 - t0) / reps, (t2 - t1) / reps
    return {"sims": len(ns), "n_total": int(np.sum(ns)), "n_min": int(np.min(ns)), "n_max": int(np.max(ns)),
            "one_by_one_ms": one * 1e3, "batched_ms": many * 1e3, "batched_us_per_sim": many / len(ns) * 1e6,
            "speedup": one / many}


def rebuild_batch_main(argv=None):
    """--rebuild-batch K: K sizes log-uniform in [--n-min, --n-max] (seeded),
    or K copies of --n."""
    import numpy as np
    from . import HH_FP64, HH_MIXED
    p = argparse.ArgumentParser()
    p.add_argument("--rebuild-batch", type=int, required=True)
    p.add_argument("--n", type=int, default=0, help="one size for all (0: log-uniform sizes)")
    p.add_argument("--n-min", type=int, default=1024)
    p.add_argument("--n-max", type=int, default=32768)
    p.add_argument("--form", default="mixed", choices=["fp64", "mixed"])
    p.add_argument("--reps", type=int, default=5)
    p.add_argument("--warm", type=int, default=2)
    a = p.parse_args(argv)
    k = a.rebuild_batch
    if a.n:
        ns = [a.n] * k
    else:
        rng = np.random.default_rng(0)
        ns = np.exp(rng.uniform(np.log(a.n_min), np.log(a.n_max), k)).astype(int).tolist()
    r = rebuild_batch(ns, HH_FP64 if a.form == "fp64" else HH_MIXED, a.reps, a.warm)
    print(json.dumps(r), flush=True)
    return r


def main(argv=None):
    import sys
    args = argv if argv is not None else sys.argv[1:]
    if "--step-profile" in args:
        step_profile_main(argv)
        return 0
    if "--list-runs" in args:
        list_runs_main(argv)
        return 0
    if "--rebuild-batch" in args:
        rebuild_batch_main(argv)
        return 0
    from . import HH_FP64, HH_MIXED

    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--n", type=int, nargs="+", default=[65536, 262144])
    p.add_argument("--theta", type=float, nargs="+", default=[0.75, 0.5, 0.3])
    p.add_argument("--n-crit", type=int, nargs="+", default=[64, 4000])
    p.add_argument("--forms", nargs="+", default=["fp64", "mixed"], choices=["fp64", "mixed"])
    p.add_argument("--intervals", type=int, default=2)
    p.add_argument("--warm", type=int, default=1)
    p.add_argument("--out", default=".")
    p.add_argument("--sweep-n", type=int, default=65536, help="N of the controlled n_i sweep (0: skip)")
    p.add_argument("--equiv-n", type=int, default=65536,
                   help="N of the equivalent-performance comparison with direct Hermite (0: skip)")
    a = p.parse_args(argv)
    sweep, sweep_fits = [], {}
    if a.sweep_n:
        for form in a.forms:
            P = HH_FP64 if form == "fp64" else HH_MIXED
            part = sweep_n_i(a.sweep_n, 0.5, 4000, P)
            sweep += part
            sweep_fits[form] = fit_force_model(part)
            for r in part:
                print(json.dumps(r), flush=True)
    equiv = []
    if a.equiv_n:
        for form in a.forms:
            e = equivalent_performance(a.equiv_n, HH_FP64 if form == "fp64" else HH_MIXED)
            equiv.append(e)
            print(json.dumps(e), flush=True)
    rows = []
    for form in a.forms:
        for n in a.n:
            for th in a.theta:
                for nc in a.n_crit:
                    r = measure(n, th, nc, HH_FP64 if form == "fp64" else HH_MIXED, a.intervals, a.warm)
                    rows.append(r)
                    print(json.dumps(r), flush=True)
    fits = {form: fit_force_model([r for r in rows if r["form"] == form]) for form in a.forms if rows}
    os.makedirs(a.out, exist_ok=True)
    with open(os.path.join(a.out, "perfmodel.json"), "w") as f:
        json.dump({"rows": rows, "fits": fits, "sweep": sweep, "sweep_fits": sweep_fits, "equiv": equiv}, f, indent=1)
    with open(os.path.join(a.out, "perfmodel.md"), "w") as f:
        if sweep:
            f.write(sweep_markdown(sweep, sweep_fits) + "\n")
        if equiv:
            f.write("Equivalent performance (Eq. 1), tree theta 0.5 against direct Hermite (theta 0) over the same "
                    "interval:\n\n| form | N | S (Tflops, 57 flop) | tree / direct time | direct steps / tree steps | "
                    "direct interactions/s |\n|---|---:|---:|---:|---:|---:|\n")
            for e in equiv:
                f.write(f"| {e['form']} | {e['n']} | {e['S_tree_tflops']:.2f} | 1/{e['speedup_over_direct']:.1f} | "
                        f"{e['steps_ratio_direct_over_tree']:.3f} | {e['direct_interactions_per_s']:.3e} |\n")
            f.write("\n")
        f.write(table_markdown(rows, fits))
    print(json.dumps({"fits": fits, "sweep_fits": sweep_fits}), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
