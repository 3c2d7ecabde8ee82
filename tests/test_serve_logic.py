"""Host logic of the continuous-batching server, with fake GPU objects (no GPU).

The fakes stand in for libhh's Context and Batch: each fake simulation needs a
fixed number of block steps per tree interval, and the fake batch keeps a
resident set with the semantics include/hh.h gives hh_batch_admit (slots and a
byte budget), hh_batch_step (one launch over the running residents, rebuilds at
each interval end, each finished simulation reported once) and
hh_batch_retire.  The checks: memory in use never exceeds the budget, requests
are admitted in arrival order as memory frees up, every request finishes
exactly once at its end time, launches mix simulations of different sizes, and
a particle cap per launch bounds the work of every launch.
"""
import numpy as np
import pytest

try:
    import paper_1602_02832_gb300 as hh
    from paper_1602_02832_gb300 import serve
except ImportError:  # libhh not built in this checkout
    hh = serve = None

pytestmark = pytest.mark.skipif(serve is None, reason="libhh.so not built")


class _Handle:
    def __init__(self, obj):
        self.value = id(obj)


class FakeCtx:
    live = 0
    peak = 0

    def __init__(self, cfg, n_max=1, nj_max=1, list_max=1, groups_max=1, device=0):
        self.n = n_max
        self.h = _Handle(self)
        self.device_bytes = 1000 * n_max
        self.t = 0.0
        self.steps_per_interval = 3 + n_max % 5
        self.done_steps = 0
        self.rebuilds = 0
        FakeCtx.live += 1
        FakeCtx.peak = max(FakeCtx.peak, FakeCtx.live)

    def hh_load_particles(self, x, v, m):
        self.x = x.copy()

    def hh_set_rebuild_device(self, on):
        self.rebuild_device = bool(on)

    def hh_run(self, t0, t1):
        self.t = t0

    def hh_rebuild(self, t):
        assert abs(t - self.t) < 1e-15
        self.rebuilds += 1

    def hh_get_state(self):
        return {"x": self.x, "v": self.x * 0}

    def hh_get_ids(self):
        return np.arange(self.n)

    def hh_get_counters(self):
        return {"block_steps": self.done_steps, "particle_steps": self.done_steps * self.n, "interactions": 7}

    def close(self):
        FakeCtx.live -= 1


class FakeBatch:
    """Resident set as include/hh.h describes it, advancing FakeCtx objects."""

    def __init__(self, precision, max_sims, max_steps, device=0):
        self.calls = []      # simulations launched per call
        self.particles = []  # particles launched per call
        self.max_sims, self.max_steps = max_sims, max_steps
        self.res = []        # [ctx, t_end, t_stop, state]
        self.budget = self.cap = 0
        self.rr = 0
        self.peak_bytes = 0

    def hh_batch_set_budget(self, budget_bytes=0, launch_particles=0):
        self.budget, self.cap = budget_bytes, launch_particles

    def _used(self):
        return sum(r[0].device_bytes for r in self.res)

    def hh_batch_admit(self, ctx, t_end):
        if len(self.res) >= self.max_sims or (self.budget and self._used() + ctx.device_bytes > self.budget):
            return False
        self.res.append([ctx, t_end, min(ctx.t + 1 / 64, t_end), 0])
        self.peak_bytes = max(self.peak_bytes, self._used())
        return True

    def hh_batch_step(self, max_steps=None):
        max_steps = max_steps or self.max_steps
        R = len(self.res)
        pick, parts = [], 0
        for q in range(R):
            r = self.res[(self.rr + q) % R]
            if r[3] != 0:
                continue
            if self.cap and pick and parts + r[0].n > self.cap:
                break
            pick.append((self.rr + q) % R)
            parts += r[0].n
        if pick:
            self.rr = (pick[-1] + 1) % R
            self.calls.append(len(pick))
            self.particles.append(parts)
            for i in pick:
                r = self.res[i]
                c, ts = r[0], r[2]
                k = 0
                while k < max_steps and c.t < ts:
                    c.done_steps += 1
                    k += 1
                    if c.done_steps % c.steps_per_interval == 0:
                        c.t = ts
                if c.t >= ts:
                    if ts >= r[1]:
                        r[3] = 1
                    else:
                        c.hh_rebuild(ts)
                        r[2] = min(ts + 1 / 64, r[1])
        done = []
        for r in self.res:
            if r[3] == 1:
                done.append(r[0].h.value)
                r[3] = 3
        # per global step: predict + select, force (+ corrector), an empty third phase
        n = max_steps if pick else 0
        self.last_phase_us = np.tile([0.25, 0.75, 0.0], (n, 1))
        return n, len(pick), done, np.ones(n)

    def hh_batch_retire(self, ctx):
        for q, r in enumerate(self.res):
            if r[0] is ctx:
                del self.res[q]
                if self.rr > q:
                    self.rr -= 1
                return
        raise AssertionError("retire of a context that is not resident")

    def hh_batch_resident(self):
        return len(self.res), sum(r[3] == 0 for r in self.res), self._used()

    def close(self):
        pass


def test_server_budget_order_and_completion(monkeypatch):
    monkeypatch.setattr(serve, "Context", FakeCtx)
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    monkeypatch.setattr(serve.Server, "estimate_bytes",
                        lambda self, r: (1000 * len(r.m), dict(n_max=len(r.m), nj_max=1, list_max=1, groups_max=1)))
    FakeCtx.live = FakeCtx.peak = 0
    sizes = [100, 700, 300, 900, 200, 500, 800, 400]
    reqs = [serve.SimRequest(i, np.zeros((n, 3)) + i, np.zeros((n, 3)), np.ones(n) / n,
                             t_end=(1 + i % 3) / 64, arrival_s=0.0) for i, n in enumerate(sizes)]
    srv = serve.Server(budget_bytes=1000 * 1500, max_sims=8, max_steps=2, rebuild_threads=2)
    res, stats = srv.run(reqs, realtime=False)
    srv.close()
    assert sorted(r.rid for r in res) == list(range(len(sizes)))
    for r in res:
        assert np.all(r.x == r.rid)  # each result belongs to its own request
        assert r.t_end == (1 + r.rid % 3) / 64
    assert FakeCtx.live == 0
    assert srv.used_bytes == 0
    # never more resident than the budget allows (1500 units, sizes as above)
    assert FakeCtx.peak <= 4
    assert srv.batch.peak_bytes <= 1000 * 1500
    assert max(srv.batch.calls) >= 2  # simulations were batched together
    assert stats.launches == len(srv.batch.calls) == len(stats.queue)
    # every launch sampled the queue: (wall s, waiting, resident), resident >= 1
    assert all(w >= 0 and r >= 1 for _, w, r in stats.queue)
    assert [t for t, _, _ in stats.queue] == sorted(t for t, _, _ in stats.queue)
    # the device-time split adds up the kernel's phases over every launch
    assert stats.phase_us[0] == pytest.approx(0.25 * len(stats.step_us))
    assert stats.phase_us[1] == pytest.approx(0.75 * len(stats.step_us))


def test_server_rejects_a_request_above_the_budget(monkeypatch):
    monkeypatch.setattr(serve, "Context", FakeCtx)
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    monkeypatch.setattr(serve.Server, "estimate_bytes",
                        lambda self, r: (1000 * len(r.m), dict(n_max=len(r.m), nj_max=1, list_max=1, groups_max=1)))
    srv = serve.Server(budget_bytes=1000 * 10, max_sims=4, max_steps=2)
    req = serve.SimRequest(0, np.zeros((50, 3)), np.zeros((50, 3)), np.ones(50) / 50, t_end=1 / 64)
    with pytest.raises(MemoryError):
        srv.run([req], realtime=False)
    srv.close()


class FakeCtxFewGroups(FakeCtx):
    """Fails its first tree build when groups_max is below n (as a device
    rebuild does with HH_ENOMEM when the tree has more groups than room)."""
    created = []

    def __init__(self, cfg, n_max=1, nj_max=1, list_max=1, groups_max=1, device=0):
        super().__init__(cfg, n_max, nj_max, list_max, groups_max, device)
        self.caps = dict(n_max=n_max, nj_max=nj_max, list_max=list_max, groups_max=groups_max)
        FakeCtxFewGroups.created.append(self.caps)

    def hh_run(self, t0, t1):
        if self.caps["groups_max"] < self.n:
            raise hh.HHError(hh.HH_ENOMEM, "hh_rebuild: more groups than groups_max")
        super().hh_run(t0, t1)


def test_admission_retries_with_bound_capacities(monkeypatch):
    # with device rebuilds the server sizes groups at n/4 without building a
    # tree; a rebuild that finds more groups fails with HH_ENOMEM and the
    # request is admitted again with the bounds themselves (groups n, j 3n)
    monkeypatch.setattr(serve, "Context", FakeCtxFewGroups)
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    FakeCtx.live = FakeCtx.peak = 0
    FakeCtxFewGroups.created = []
    n = 400
    req = serve.SimRequest(0, np.zeros((n, 3)), np.zeros((n, 3)), np.ones(n) / n, t_end=1 / 64)
    srv = serve.Server(budget_bytes=10 ** 9, max_sims=2, max_steps=4, rebuild_device=True)
    est, caps = srv.estimate_bytes(req)
    assert caps["groups_max"] < n and caps["nj_max"] == 2 * n + 64 and est > 0
    res, _ = srv.run([req], realtime=False)
    srv.close()
    assert [c["groups_max"] for c in FakeCtxFewGroups.created] == [caps["groups_max"], n]
    assert FakeCtxFewGroups.created[1]["nj_max"] == 3 * n + 64
    assert len(res) == 1 and FakeCtx.live == 0 and srv.used_bytes == 0


def test_admission_error_other_than_memory_is_raised(monkeypatch):
    class FakeCtxBad(FakeCtx):
        def hh_run(self, t0, t1):
            raise hh.HHError(hh.HH_EINVAL, "bad particles")

    monkeypatch.setattr(serve, "Context", FakeCtxBad)
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    FakeCtx.live = 0
    req = serve.SimRequest(0, np.zeros((10, 3)), np.zeros((10, 3)), np.ones(10) / 10, t_end=1 / 64)
    srv = serve.Server(budget_bytes=10 ** 9, max_sims=2, max_steps=4, rebuild_device=True)
    with pytest.raises(hh.HHError):
        srv.run([req], realtime=False)
    srv.close()
    assert FakeCtx.live == 0


def test_particle_cap_bounds_every_launch_and_all_finish(monkeypatch):
    # launch_particles: each launch advances at most that many particles (at
    # least one simulation), round robin, and every request still finishes
    monkeypatch.setattr(serve, "Context", FakeCtx)
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    monkeypatch.setattr(serve.Server, "estimate_bytes",
                        lambda self, r: (1000 * len(r.m), dict(n_max=len(r.m), nj_max=1, list_max=1, groups_max=1)))
    FakeCtx.live = FakeCtx.peak = 0
    sizes = [100, 700, 300, 900, 200, 500, 800, 400]
    reqs = [serve.SimRequest(i, np.zeros((n, 3)) + i, np.zeros((n, 3)), np.ones(n) / n,
                             t_end=(1 + i % 3) / 64, arrival_s=0.0) for i, n in enumerate(sizes)]
    srv = serve.Server(budget_bytes=10 ** 9, max_sims=8, max_steps=2, launch_particles=1000)
    res, stats = srv.run(reqs, realtime=False)
    srv.close()
    assert sorted(r.rid for r in res) == list(range(len(sizes)))
    assert all(p <= 1000 or c == 1 for p, c in zip(srv.batch.particles, srv.batch.calls))
    assert max(srv.batch.particles) <= max(1000, max(sizes))
    assert FakeCtx.live == 0 and srv.used_bytes == 0
