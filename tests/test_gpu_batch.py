"""Batched persistent block steps (hh_batch_run) against single-simulation runs.

Every simulation of a batch must give the same state as when it runs alone
through hh_advance (same tiles, active masks and list parts; fixed-order
sums), whatever else shares the launch and however the run is cut into
launches.  With step-adaptive list parts (work_split > 0, the batched loop
only) the reference is the simulation alone in a batch.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hh():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1602_02832_gb300 as hh
    return hh


def _ctx(hh, prec, n, seed, theta, n_crit=32, salpeter=False):
    x, v, m = (synth.plummer_salpeter if salpeter else synth.plummer)(n, seed)
    c = hh.hh_config_default()
    c.eps2 = 1e-6
    c.precision = prec
    c.theta = theta
    c.n_crit = n_crit
    ctx = hh.Context(c, n, 2 * n, 64 * n * max(1, n // 16), n)
    ctx.hh_load_particles(x.T, v.T, m)
    ctx.hh_run(0.0, 0.0)
    return ctx


SPECS = [(600, 1, 0.5, False), (1500, 2, 0.3, True), (300, 3, 0.7, False), (1024, 4, 0.5, True)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_equals_alone(hh, prec):
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    t1 = 2.0 ** -6
    alone = []
    for n, seed, th, sal in SPECS:
        with _ctx(hh, P, n, seed, th, salpeter=sal) as c:
            c.hh_advance(t1)
            alone.append((c.hh_get_state(), c.hh_get_counters()))
    ctxs = [_ctx(hh, P, n, seed, th, salpeter=sal) for n, seed, th, sal in SPECS]
    with hh.Batch(P, max_sims=8, max_steps=4096) as b:
        steps, tn, us = b.hh_batch_run(ctxs, [t1] * len(ctxs))
    assert np.all(tn > t1) and steps > 0 and len(us) == steps and np.all(us > 0)
    for c, (st, cnt) in zip(ctxs, alone):
        got = c.hh_get_state()
        gc = c.hh_get_counters()
        for k in ("x", "v", "a", "jk", "t", "dt"):
            assert np.array_equal(got[k], st[k]), k
        assert gc["block_steps"] == cnt["block_steps"]
        assert gc["particle_steps"] == cnt["particle_steps"]
        assert gc["interactions"] == cnt["interactions"]
        c.close()
    assert steps == max(c[1]["block_steps"] for c in alone)


def test_batch_result_does_not_depend_on_cta_count(hh):
    # the same batch on every SM and on 37 of them (items land on other SMs,
    # in another order): identical states
    P = hh.HH_MIXED
    t1 = 2.0 ** -7
    states = []
    for ctas in (0, 37):
        ctxs = [_ctx(hh, P, n, seed, th, salpeter=sal) for n, seed, th, sal in SPECS]
        with hh.Batch(P, max_sims=8, max_steps=4096) as b:
            if ctas:
                b.hh_batch_set_ctas(ctas)
            b.hh_batch_run(ctxs, [t1] * len(ctxs))
        states.append([c.hh_get_state() for c in ctxs])
        for c in ctxs:
            c.close()
    for a, b_ in zip(*states):
        for k in ("x", "v", "a", "jk", "t", "dt"):
            assert np.array_equal(a[k], b_[k]), k
    with hh.Batch(P, max_sims=2, max_steps=8) as b:
        with pytest.raises(hh.HHError):
            b.hh_batch_set_ctas(100000)


def test_batch_in_short_launches_and_with_rebuilds(hh):
    # continuous batching: the same simulations advanced in launches of 7
    # global steps, rebuilt at each dt_tree, reach the same state as one
    # simulation advanced alone with hh_advance + hh_rebuild
    P = hh.HH_MIXED
    dtt = 2.0 ** -6
    ref = []
    for n, seed, th, sal in SPECS[:3]:
        with _ctx(hh, P, n, seed, th, salpeter=sal) as c:
            for k in range(2):
                c.hh_advance((k + 1) * dtt)
                c.hh_rebuild((k + 1) * dtt)
            ref.append(c.hh_get_state())
    ctxs = [_ctx(hh, P, n, seed, th, salpeter=sal) for n, seed, th, sal in SPECS[:3]]
    t_stop = np.full(3, dtt)
    with hh.Batch(P, max_sims=4, max_steps=64) as b:
        done = np.zeros(3, bool)
        rounds = 0
        while not done.all():
            live = [i for i in range(3) if not done[i]]
            steps, tn, _ = b.hh_batch_run([ctxs[i] for i in live], t_stop[live], max_steps=7)
            for i, t in zip(live, tn):
                if t > t_stop[i]:
                    ctxs[i].hh_rebuild(t_stop[i])
                    if t_stop[i] >= 2 * dtt:
                        done[i] = True
                    t_stop[i] += dtt
            rounds += 1
            assert rounds < 10000
    for c, st in zip(ctxs, ref):
        got = c.hh_get_state()
        for k in ("x", "v", "t", "dt"):
            assert np.array_equal(got[k], st[k]), k
        c.close()


def test_batch_rejects_bad_requests(hh):
    with hh.Batch(hh.HH_FP64, max_sims=2, max_steps=16) as b:
        c1 = _ctx(hh, hh.HH_FP64, 200, 5, 0.5)
        c2 = _ctx(hh, hh.HH_MIXED, 200, 6, 0.5)
        with pytest.raises(hh.HHError):
            b.hh_batch_run([c1, c2], [0.01, 0.01])  # precision mismatch
        with pytest.raises(hh.HHError):
            b.hh_batch_run([c1, c1], [0.01, 0.01])  # same context twice
        with pytest.raises(hh.HHError):
            b.hh_batch_run([c1], [0.01], max_steps=17)  # above the batch's step capacity
        steps, tn, _ = b.hh_batch_run([c1], [0.01], max_steps=16)
        assert 0 < steps <= 16
        c1.close()
        c2.close()


def test_bounded_barrier_reports_timeout(hh):
    # Failure detection without a GPU fault: a CTA that never arrives makes
    # the others' bounded waits give up; the call reports HH_ETIMEOUT and the
    # context stays usable (the normal barrier run afterwards succeeds).
    rc, t = hh.hh_barrier_selftest(skip_cta=-1)
    assert rc == hh.HH_OK and t < 1.0
    rc, t = hh.hh_barrier_selftest(skip_cta=3)
    assert rc == hh.HH_ETIMEOUT and 0.05 < t < 30.0
    rc, t = hh.hh_barrier_selftest(skip_cta=-1)
    assert rc == hh.HH_OK


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("small", [False, True])
def test_step_adaptive_parts_do_not_depend_on_the_batch(hh, prec, small):
    # work_split: equal-cost list parts only in block steps with at least 64
    # active particles; tile_j_small: short parts in steps with at most 16
    # (both counts are each simulation's own), so a simulation alone and the
    # same simulation beside others reach the same bits; the graph loop (parts
    # of tile_j throughout) agrees within FP64 reordering
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    t1 = 2.0 ** -6

    alone = []
    for n, seed, th, sal in SPECS:
        x, v, m = (synth.plummer_salpeter if sal else synth.plummer)(n, seed)
        alone.append((x, v, m, th))

    def make(x, v, m, th):
        c = hh.hh_config_default()
        c.eps2, c.precision, c.theta, c.n_crit = 1e-6, P, th, 32
        c.tile_j = 256 if P == hh.HH_FP64 else 512
        c.work_item, c.work_split = 2048, 64
        c.tile_j_small = (64 if P == hh.HH_FP64 else 128) if small else 0
        ctx = hh.Context(c, len(m), 2 * len(m), 64 * len(m) * max(1, len(m) // 16), len(m))
        ctx.hh_load_particles(x.T, v.T, m)
        ctx.hh_run(0.0, 0.0)
        return ctx

    ref = []
    for spec in alone:
        with make(*spec) as c, hh.Batch(P, max_sims=1, max_steps=4096) as b:
            b.hh_batch_run([c], [t1])
            ref.append(c.hh_get_state())
    ctxs = [make(*spec) for spec in alone]
    with hh.Batch(P, max_sims=8, max_steps=4096) as b:
        b.hh_batch_run(ctxs, [t1] * len(ctxs))
    for c, st in zip(ctxs, ref):
        got = c.hh_get_state()
        for k in ("x", "v", "a", "jk", "t", "dt"):
            assert np.array_equal(got[k], st[k]), k
        c.close()
    if P == hh.HH_FP64:
        for spec, st in zip(alone, ref):
            with make(*spec) as c:
                c.hh_advance(t1)
                g = c.hh_get_state()
            assert np.array_equal(g["t"], st["t"])
            assert np.abs(g["x"] - st["x"]).max() < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("work", [(0, 0), (8192, 0), (0, 64)])
def test_list_mode_prediction_changes_no_bit(hh, prec, work):
    # N = 2^18 (about 3.4e5 j entries, above the size from which the batched
    # loop predicts only the entries of a small step's list parts): the
    # batched run equals, bit for bit, the graph loop, which predicts every
    # entry at every step; with equal-cost parts in every step, a lone active
    # particle's part is 8192 entries long, and every entry of it is predicted
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    n = 1 << 18
    x, v, m = synth.plummer(n, 9)
    t1 = 2.0 ** -9

    def make():
        c = hh.hh_config_default()
        c.eps2, c.precision, c.n_crit = 1e-8, P, 64
        c.work_item, c.work_split = work
        z = np.zeros((3, n))
        T0 = hh.hh_tree_build(x.T, v.T, z, z, m, leaf=8, n_crit=64, theta=0.5)
        ctx = hh.Context(c, n, 2 * n, 2 * len(T0.idx) + 1024, 2 * T0.n_groups + 64)
        ctx.hh_load_particles(x.T, v.T, m)
        ctx.hh_set_rebuild_device(True)
        ctx.hh_run(0.0, 0.0)
        assert ctx.nj >= 1 << 18
        return ctx

    with make() as c:
        c.hh_advance(t1)
        ref = c.hh_get_state()
        ref_c = c.hh_get_counters()
    with make() as c, hh.Batch(P, max_sims=1, max_steps=4096) as b:
        steps, tn, _ = b.hh_batch_run([c], [t1])
        got = c.hh_get_state()
        got_c = c.hh_get_counters()
    assert tn[0] > t1 and steps > 10
    assert 0 < got_c["list_steps"] < steps and ref_c["list_steps"] == 0  # the mode was used, not always
    assert got_c["interactions"] == ref_c["interactions"]
    if work[1] > 0:
        # with work_split the batched loop splits lists otherwise than the
        # graph loop (in FP64 its small and medium steps take other parts), so
        # sums differ in their last bits; a stale prediction would not
        assert np.array_equal(got["t"], ref["t"]) and np.array_equal(got["dt"], ref["dt"])
        assert np.abs(got["x"] - ref["x"]).max() < 1e-9
        return
    for k in ("x", "v", "a", "jk", "t", "dt"):
        assert np.array_equal(got[k], ref[k]), k



@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_beyond_the_cached_descriptors(hh, prec):
    # 300 small simulations in one batch: beyond the 32 descriptors and the
    # 256 step caches a CTA keeps in shared memory, the kernel reads them
    # from global memory; every simulation still reaches its lone bits
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    t1 = 2.0 ** -8
    specs = [(64 + (k * 37) % 96, 1000 + k) for k in range(300)]

    def make(n, seed):
        x, v, m = synth.plummer(n, seed)
        c = hh.hh_config_default()
        c.eps2, c.precision, c.n_crit = 1e-6, P, 32
        ctx = hh.Context(c, n, 2 * n, 64 * n * max(1, n // 16), n)
        ctx.hh_load_particles(x.T, v.T, m)
        ctx.hh_run(0.0, 0.0)
        return ctx

    ref = []
    with hh.Batch(P, max_sims=1, max_steps=4096) as b:
        for spec in specs:
            with make(*spec) as c:
                b.hh_batch_run([c], [t1])
                ref.append(c.hh_get_state())
    ctxs = [make(*spec) for spec in specs]
    try:
        with hh.Batch(P, max_sims=len(specs), max_steps=4096) as b:
            b.hh_batch_run(ctxs, [t1] * len(ctxs))
        for c, st in zip(ctxs, ref):
            got = c.hh_get_state()
            for k in ("x", "v", "a", "jk", "t", "dt"):
                assert np.array_equal(got[k], st[k]), k
    finally:
        for c in ctxs:
            c.close()
