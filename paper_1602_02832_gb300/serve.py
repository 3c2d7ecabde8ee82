"""Continuous-batching server of cluster simulations over libhh.

Requests (independent N-body simulations with their own N, masses and end
time) are admitted while their device memory fits a budget, stay resident on
the GPU, and advance together.  Admission, launches and rebuilds are libhh's
resident set (hh_batch_admit / hh_batch_step / hh_batch_retire): every
iteration is ONE persistent batched launch that gives each running resident up
to `max_steps` block steps, stopping each at its next tree rebuild time
(Section 2: lists are rebuilt every dt_tree), followed by the rebuilds of the
simulations that reached it.  Finished simulations are read back, retired
(their memory returns to the budget) and waiting requests take their place.
With `launch_particles` a launch advances at most that many particles (round
robin over the residents), which bounds the latency of each global block step.

This module keeps only the host side: request preparation (initial conditions,
a memory estimate) and context creation (initial forces) run on worker
threads so the launches keep running meanwhile.  A simulation's result does
not depend on what else shares the launches (see hh_batch_run).
"""
from __future__ import annotations

import math
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import HH_ENOMEM, HH_MIXED, Batch, Context, HHError, hh_config_default, hh_tree_build


@dataclass
class SimRequest:
    rid: int
    x: np.ndarray | None   # [n, 3] positions (any order); None: call make()
    v: np.ndarray | None   # [n, 3]
    m: np.ndarray | None   # [n]
    t_end: float           # multiple of dt_tree
    arrival_s: float = 0.0  # offset from the stream start
    make: object = None    # optional callable returning (x, v, m), run at admission

    def materialise(self):
        if self.x is None:
            self.x, self.v, self.m = self.make()
        return self


@dataclass
class SimResult:
    rid: int
    n: int
    x: np.ndarray  # [n, 3] final state in request order
    v: np.ndarray
    t_end: float
    arrival_s: float
    admit_s: float
    done_s: float
    block_steps: int
    particle_steps: int
    interactions: int


@dataclass
class _Live:
    req: SimRequest
    ctx: Context
    bytes: int             # device bytes of the context
    admit_s: float


@dataclass
class ServerStats:
    step_us: list = field(default_factory=list)       # duration of each global block step
    live_per_step: list = field(default_factory=list)  # simulations advanced in that launch
    phase_us: list = field(default_factory=lambda: [0.0, 0.0])  # device time in predict + select, force + correct
    # per launch: (wall seconds, requests arrived but not yet resident, resident simulations)
    queue: list = field(default_factory=list)
    launches: int = 0
    block_steps: int = 0          # sum over simulations of block steps
    interactions: int = 0
    wall_s: float = 0.0


# Measured crossover for a context rebuilt alone: at N = 1024 / 2048 / 4096 a rebuild took
# 0.62 / 1.45 / 3.5 ms on the host, and 0.39 ms at N = 1024 and 0.50 ms at N = 4096 on the device
# (whose fixed cost is kernel-launch latency): callers that rebuild one context at a time use the
# device from AUTO_DEVICE_MIN_N.  The server's rebuilds run batched (hh_batch_step builds all due
# device contexts of a launch at once, 13 us a simulation for 64 at N = 1024), so its "auto" takes
# the device at every size.
AUTO_DEVICE_MIN_N = 2048


class Server:
    """Continuous batching of block steps across resident simulations."""

    def _on_device(self, n):
        return True if self.rebuild_device == "auto" else self.rebuild_device

    def __init__(self, precision=HH_MIXED, budget_bytes=150 * 10 ** 9, max_sims=256, max_steps=64,
                 eps2=1e-8, eta=0.02, theta=0.5, n_crit=64, dt_tree=2.0 ** -6, rebuild_threads=4, device=0,
                 rebuild_device=False, order=0, launch_particles=0, tile_i=0, tile_j=0, work_item=0, work_split=0):
        self.precision = precision
        # True / False, or "auto": the device builder (batched rebuilds make
        # it the faster one at every size)
        self.rebuild_device = rebuild_device if rebuild_device == "auto" else bool(rebuild_device)
        self.budget = int(budget_bytes)
        self.max_sims = int(max_sims)
        self.max_steps = int(max_steps)
        self.launch_particles = int(launch_particles)
        self.device = device
        self.cfg = hh_config_default()
        self.cfg.eps2, self.cfg.eta, self.cfg.theta, self.cfg.n_crit = eps2, eta, theta, n_crit
        self.cfg.dt_max = dt_tree
        self.cfg.dt_tree = dt_tree
        self.cfg.precision = precision
        self.cfg.order = order
        # list decomposition (0: the library's defaults); see hh_config
        self.cfg.tile_i = tile_i or self.cfg.tile_i
        self.cfg.tile_j = tile_j
        self.cfg.work_item = work_item
        self.cfg.work_split = work_split
        self.batch = Batch(precision, max_sims=max_sims, max_steps=max_steps, device=device)
        self.batch.hh_batch_set_budget(self.budget, self.launch_particles)
        self.pool = ThreadPoolExecutor(max_workers=rebuild_threads)
        self.stats = ServerStats()
        self._reserved = 0  # estimated bytes of contexts created but not yet resident

    @property
    def used_bytes(self):
        """Device bytes held by resident contexts plus those being created."""
        return self.batch.hh_batch_resident()[2] + self._reserved

    def close(self):
        self.pool.shutdown(wait=True)
        self.batch.close()

    # -- admission ---------------------------------------------------------
    def estimate_bytes(self, req: SimRequest) -> tuple[int, dict]:
        """Device bytes a simulation needs and the capacities to create it with.
        With device rebuilds no tree is built here: j entries get 2n, groups n/4
        (admission retries with n if a rebuild finds more), the list buffer
        starts small and the first device rebuild grows it to the need; the byte estimate (used only until the
        context reports its own size) takes a list length above those measured
        for Plummer spheres.  With host rebuilds the capacities come from a host
        build of the tree."""
        n = len(req.m)
        if self._on_device(n):
            th = max(self.cfg.theta, 0.05)
            per = min(2.0 * n, 400.0 * (0.5 / th) ** 2)  # list entries per particle, generous
            caps = dict(n_max=n, nj_max=2 * n + 64, list_max=16 * n + 4096, groups_max=n // 4 + 64)
            L_est = int(per * n) + 4096
        else:
            z = np.zeros((3, n))
            T = hh_tree_build(req.x.T, req.v.T, z, z, req.m, leaf=8, n_crit=self.cfg.n_crit, theta=self.cfg.theta)
            caps = dict(n_max=n, nj_max=n + 2 * T.n_nodes + 64, list_max=int(1.5 * len(T.idx)) + 4096,
                        groups_max=2 * T.n_groups + 64)
            L_est = caps["list_max"]
        nj, L, G = caps["nj_max"], L_est, caps["groups_max"]
        rec = 48 if self.precision == HH_MIXED else 64
        est = (nj * (14 * 8 + rec) + n * (8 * 8 + 4 * 3 + 7 * 8) + L * 4 + G * 8
               + (n // 32 + G) * (16 + 4 + 16 + 32 * 56) * 2)
        return int(est), caps

    def _create(self, req: SimRequest, caps: dict, now_s: float) -> _Live:
        """Context with the request's particles, tree, initial forces and steps
        (not yet resident)."""
        for attempt in range(2):
            ctx = Context(self.cfg, device=self.device, **caps)
            try:
                ctx.hh_load_particles(np.ascontiguousarray(req.x.T), np.ascontiguousarray(req.v.T), req.m)
                ctx.hh_set_rebuild_device(self._on_device(len(req.m)))
                ctx.hh_run(0.0, 0.0)  # tree, initial forces, node derivatives, initial steps
                break
            except HHError as e:
                ctx.close()
                if e.code != HH_ENOMEM or attempt:
                    raise
                n = caps["n_max"]  # more groups or cells than guessed: the bounds themselves
                caps = dict(caps, nj_max=3 * n + 64, groups_max=n)
        return _Live(req, ctx, ctx.device_bytes, now_s)

    def _finish(self, s: _Live, now_s: float) -> SimResult:
        st = s.ctx.hh_get_state()
        ids = s.ctx.hh_get_ids()
        c = s.ctx.hh_get_counters()
        n = len(s.req.m)
        x = np.zeros((n, 3))
        v = np.zeros((n, 3))
        x[ids] = st["x"].T
        v[ids] = st["v"].T
        s.ctx.close()
        return SimResult(s.req.rid, n, x, v, s.req.t_end, s.req.arrival_s, s.admit_s, now_s, c["block_steps"],
                         c["particle_steps"], c["interactions"])

    # -- main loop ---------------------------------------------------------
    def run(self, requests: list[SimRequest], realtime: bool = True, max_wall_s: float = math.inf):
        """Serves the requests (sorted by arrival); returns (results, stats).
        With realtime, a request becomes visible at its arrival offset.
        Preparation (initial conditions, memory estimate) and context creation
        (initial forces) run on the worker threads; contexts are admitted to
        the batch's resident set in arrival order as slots and budget allow."""
        pending = sorted(requests, key=lambda r: r.arrival_s)
        preparing = []                                   # futures -> (req, est, caps)
        waiting: list[tuple[SimRequest, int, dict]] = []  # prepared, in arrival order
        creating = []                                    # (future -> _Live, estimated bytes)
        created: list[_Live] = []                        # not yet admitted, in order
        live: dict[int, _Live] = {}                      # resident, by context handle
        results: list[SimResult] = []
        t0 = time.perf_counter()

        def prepare(r):
            r.materialise()
            est, caps = self.estimate_bytes(r)
            return r, est, caps

        def create(r, caps):
            return self._create(r, caps, time.perf_counter() - t0)

        try:
            while pending or preparing or waiting or creating or created or live:
                now = time.perf_counter() - t0
                if now > max_wall_s:
                    break
                while pending and (not realtime or pending[0].arrival_s <= now):
                    preparing.append(self.pool.submit(prepare, pending.pop(0)))
                # prepared requests join the queue in arrival order
                while preparing and preparing[0].done():
                    waiting.append(preparing.pop(0).result())
                # contexts are created while slots and the estimated memory allow
                held = self.batch.hh_batch_resident()[2]
                while (waiting and len(live) + len(creating) + len(created) < self.max_sims
                       and held + self._reserved + waiting[0][1] <= self.budget):
                    r, est, caps = waiting.pop(0)
                    self._reserved += est
                    creating.append((self.pool.submit(create, r, caps), est))
                if waiting and not (live or creating or created) and waiting[0][1] > self.budget:
                    raise MemoryError(f"request {waiting[0][0].rid} needs {waiting[0][1]} bytes, above the budget")
                while creating and creating[0][0].done():
                    f, est = creating.pop(0)
                    self._reserved -= est
                    s = f.result()
                    self._reserved += s.bytes
                    created.append(s)
                # admission by the contexts' measured bytes (libhh's resident set)
                while created and self.batch.hh_batch_admit(created[0].ctx, created[0].req.t_end):
                    s = created.pop(0)
                    self._reserved -= s.bytes
                    live[s.ctx.h.value] = s
                if created and not live and not creating:
                    raise MemoryError(f"request {created[0].req.rid} needs {created[0].bytes} bytes, above the budget")
                if not live:
                    busy = [x[0] for x in creating] + preparing
                    if busy:
                        busy[0].result()
                    elif pending and realtime:
                        time.sleep(max(0.0, min(0.01, pending[0].arrival_s - (time.perf_counter() - t0))))
                    continue
                steps, launched, done, us = self.batch.hh_batch_step(self.max_steps)
                if launched:
                    self.stats.queue.append((time.perf_counter() - t0,
                                             len(preparing) + len(waiting) + len(creating) + len(created), len(live)))
                    self.stats.launches += 1
                    self.stats.step_us.extend(us.tolist())
                    self.stats.live_per_step.extend([launched] * len(us))
                    ph = getattr(self.batch, "last_phase_us", None)
                    if ph is not None and len(ph):
                        self.stats.phase_us[0] += float(ph[:, 0].sum())
                        self.stats.phase_us[1] += float(ph[:, 1].sum() + ph[:, 2].sum())
                for h in done:
                    s = live.pop(h)
                    self.batch.hh_batch_retire(s.ctx)
                    res = self._finish(s, time.perf_counter() - t0)
                    self.stats.block_steps += res.block_steps
                    self.stats.interactions += res.interactions
                    results.append(res)
        finally:
            for f in preparing:
                f.result()
            for f, est in creating:
                s = f.result()
                self._reserved -= est
                s.ctx.close()
            for s in created:
                self._reserved -= s.bytes
                s.ctx.close()
            for s in live.values():  # stopped by max_wall_s (or an error)
                c = s.ctx.hh_get_counters()
                self.stats.block_steps += c["block_steps"]
                self.stats.interactions += c["interactions"]
                self.batch.hh_batch_retire(s.ctx)
                s.ctx.close()
        self.stats.wall_s = time.perf_counter() - t0
        return results, self.stats


def latency_summary(step_us) -> dict:
    if not len(step_us):
        return {"p50": None, "p99": None, "n": 0}
    u = np.asarray(step_us, dtype=np.float64)
    return {"p50": float(np.quantile(u, 0.5)), "p99": float(np.quantile(u, 0.99)), "n": int(u.size)}
