"""Batched device rebuilds (hh_batch_rebuild, and hh_batch_step through it):
the tree-loop step 1 of Section 2 for many contexts at once, each builder
step one launch over all of them.  Every context must end with the particle
order, groups, lists and node records (all j entries, bit for bit) that
hh_rebuild gives it alone, whatever else is in the batch: contexts of other
sizes, orders, opening angles and group sizes, a first build (no depth guess)
beside later ones, a tree deeper than the last one, and contexts whose
rebuild fails; and block steps from a batched build's lists, node records and
(mixed form) base records give the bits of those from a build alone."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

# (n, seed, salpeter, theta, n_crit, order)
SPECS = [(2, 1, False, 0.5, 64, "morton"),
         (9, 2, False, 0.5, 8, "morton"),
         (700, 3, True, 0.0, 32, "morton"),
         (3000, 4, False, 0.5, 64, "hilbert"),
         (5000, 5, True, 0.3, 256, "morton"),
         (20000, 6, False, 0.7, 64, "morton"),
         (1500, 7, False, 0.5, 16, "hilbert"),
         (40000, 8, False, 0.5, 64, "morton")]  # above the batched builder's size: rebuilt alone


@pytest.fixture(scope="module")
def hh():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1602_02832_gb300 as hh
    return hh


def _ctx(hh, n, theta, n_crit, order, x, v, m, cells=None, prec=None):
    cfg = hh.hh_config_default()
    cfg.eps2, cfg.theta, cfg.n_crit = 1e-6, theta, n_crit
    if prec is not None:
        cfg.precision = prec
    cfg.order = hh.HH_ORDER_HILBERT if order == "hilbert" else hh.HH_ORDER_MORTON
    # (the list buffer starts small: a device rebuild grows it to the need)
    ctx = hh.Context(cfg, n, n + (2 * n + 64 if cells is None else cells), 64 * n + 4096, n + 64)
    ctx.hh_load_particles(x.T, v.T, m)
    ctx.hh_set_rebuild_device(True)
    return ctx


def _snap(ctx):
    n = len(ctx.hh_get_ids())
    off, idx, gof = ctx.hh_get_lists()
    return {"ids": ctx.hh_get_ids(), "off": off, "idx": idx, "gof": gof, "j": ctx.hh_get_j(0, ctx.nj),
            "nj": ctx.nj, "n": n}


def _same(a, b):
    assert a["nj"] == b["nj"]
    for k in ("ids", "off", "idx", "gof"):
        assert np.array_equal(a[k], b[k]), k
    for k, u in a["j"].items():
        assert np.array_equal(u, b["j"][k]), k


def _inputs(spec):
    n, seed, sal, *_ = spec
    return (synth.plummer_salpeter if sal else synth.plummer)(n, seed)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_rebuild_equals_alone(hh, prec):
    # Each context is rebuilt twice at t = 0 from its own forces and steps
    # (hh_run), once alone and once in a batched build; then a stretch of
    # block steps runs from the rebuilt lists and node records (and, mixed,
    # the base records the batched build's closing kernel refreshed).
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    alone, many = [], []
    for s in SPECS:
        x, v, m = _inputs(s)
        alone.append(_ctx(hh, s[0], s[3], s[4], s[5], x, v, m, prec=P))
        many.append(_ctx(hh, s[0], s[3], s[4], s[5], x, v, m, prec=P))
    for c in alone + many:
        c.hh_run(0.0, 0.0)
    with hh.Batch(P, max_sims=len(SPECS), max_steps=8) as b:
        for rep in range(2):
            for c in alone:
                c.hh_rebuild(0.0)
            assert b.hh_batch_rebuild(many, 0.0) == [hh.HH_OK] * len(SPECS)
            for c, d in zip(alone, many):
                _same(_snap(c), _snap(d))
        _, tn, _ = b.hh_batch_run(alone, 2.0 ** -6)
        _, tm, _ = b.hh_batch_run(many, 2.0 ** -6)
        assert np.array_equal(tn, tm)
        for c, d in zip(alone, many):
            sa, sb = c.hh_get_state(), d.hh_get_state()
            for k in sa:
                assert np.array_equal(sa[k], sb[k]), k
    for c in alone + many:
        c.close()


def test_batched_rebuild_of_a_deeper_tree_and_of_failing_contexts(hh):
    # context 0: a uniform cube, then a Plummer sphere (deeper than the depth
    # guess); context 1: room for 10 cells (HH_ENOMEM); context 2: particles
    # not at the rebuild time (HH_ESTATE); context 3: a host builder (rebuilt
    # alone, in the same call)
    n = 20000
    rng = np.random.default_rng(5)
    xu = rng.uniform(-1.0, 1.0, size=(n, 3))
    x, v, m = synth.plummer(n, 43)
    x1, v1, m1 = synth.plummer(2000, 47)
    x3, v3, m3 = synth.plummer(1000, 48)
    ref = _ctx(hh, n, 0.5, 64, "morton", xu, v, m)
    ref.hh_rebuild(0.0)
    ref.hh_load_particles(x.T, v.T, m)
    ref.hh_rebuild(0.0)
    want = _snap(ref)
    ref3 = _ctx(hh, 1000, 0.5, 64, "morton", x3, v3, m3)
    ref3.hh_set_rebuild_device(False)
    ref3.hh_rebuild(0.0)
    want3 = _snap(ref3)
    c0 = _ctx(hh, n, 0.5, 64, "morton", xu, v, m)
    c1 = _ctx(hh, 2000, 0.5, 64, "morton", x1, v1, m1, cells=10)
    c2 = _ctx(hh, 2000, 0.5, 64, "morton", x1, v1, m1)
    c3 = _ctx(hh, 1000, 0.5, 64, "morton", x3, v3, m3)
    c3.hh_set_rebuild_device(False)
    with hh.Batch(hh.HH_FP64, max_sims=4, max_steps=8) as b:
        assert b.hh_batch_rebuild([c0], 0.0) == [hh.HH_OK]
        c0.hh_load_particles(x.T, v.T, m)
        rcs = b.hh_batch_rebuild([c0, c1, c2, c3], [0.0, 0.0, 0.5, 0.0], check=False)
        assert rcs == [hh.HH_OK, hh.HH_ENOMEM, hh.HH_ESTATE, hh.HH_OK]
        assert "nj_max" in hh.hh_last_error(c1.h) and "synchronised" in hh.hh_last_error(c2.h)
        with pytest.raises(hh.HHError) as e:  # the first failure is the call's result
            b.hh_batch_rebuild([c1, c0], 0.0)
        assert e.value.code == hh.HH_ENOMEM
        with pytest.raises(hh.HHError) as e:
            b.hh_batch_rebuild([c0, c0], 0.0)
        assert e.value.code == hh.HH_EINVAL
    _same(want, _snap(c0))
    _same(want3, _snap(c3))
    for c in (c1, c2):
        with pytest.raises(hh.HHError) as e2:  # no valid lists after a failed rebuild
            c.hh_step()
        assert e2.value.code == hh.HH_ESTATE
    st = c1.hh_get_state()  # the failed build reordered nothing
    assert np.array_equal(st["x"], np.ascontiguousarray(x1.T))
    for c in (ref, ref3, c0, c1, c2, c3):
        c.close()


def test_perfmodel_times_batched_rebuilds(hh):
    from paper_1602_02832_gb300 import perfmodel
    r = perfmodel.rebuild_batch([1024, 3000, 700, 5000], hh.HH_MIXED, reps=1, warm=1)
    assert r["sims"] == 4 and r["n_total"] == 9724
    assert r["one_by_one_ms"] > 0 and r["batched_ms"] > 0 and r["speedup"] > 0
