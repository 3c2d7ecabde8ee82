"""Tree, groups and lists built on the device (hh_set_rebuild_device) against
the oracle's builder on the same positions.  Both follow the same rules; the
device sums node moments in another order, so a node's centre of mass may
differ in the last bits and, very rarely, flip an opening decision at a tie."""
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


@pytest.mark.parametrize("n,theta,n_crit,salp,order", [(3000, 0.5, 64, False, "morton"),
                                                       (20000, 0.3, 256, True, "morton"),
                                                       (777, 0.0, 32, False, "morton"),
                                                       (65536, 0.5, 64, False, "morton"),
                                                       (3000, 0.5, 64, True, "hilbert"),
                                                       (65536, 0.5, 64, False, "hilbert")])
def test_device_tree_matches_oracle(hh, orc, n, theta, n_crit, salp, order):
    x, v, m = (synth.plummer_salpeter if salp else synth.plummer)(n, 41)
    cfg = hh.hh_config_default()
    cfg.theta, cfg.n_crit = theta, n_crit
    cfg.order = hh.HH_ORDER_HILBERT if order == "hilbert" else hh.HH_ORDER_MORTON
    z = np.zeros_like(x)
    T = orc.tree_build(x, v, z, z, m, leaf=8, n_crit=n_crit, theta=theta, order=order)
    with hh.Context(cfg, n, n + 2 * T.n_cells + 64, 2 * len(T.list_idx) + 1024, 2 * T.n_groups + 64) as ctx:
        ctx.hh_load_particles(x.T, v.T, m)
        ctx.hh_set_rebuild_device(True)
        ctx.hh_rebuild(0.0)
        ids = ctx.hh_get_ids()
        off, idx, gof = ctx.hh_get_lists()
        nodes = ctx.hh_get_j(n, ctx.nj - n)
    assert np.array_equal(ids, T.perm)                 # Morton order (keys and tie order)
    assert ctx is not None and len(off) - 1 == T.n_groups
    assert np.array_equal(gof, T.group_of)
    np.testing.assert_allclose(nodes["m"], T.node_m, rtol=1e-13)
    np.testing.assert_allclose(nodes["x"].T, T.node_x, rtol=1e-12, atol=1e-14)
    same = np.array_equal(off, T.list_off) and np.array_equal(idx, T.list_idx)
    if not same:  # only rare tie flips are acceptable
        diff = sum(1 for g in range(T.n_groups)
                   if not np.array_equal(idx[off[g]:off[g + 1]], T.list_idx[T.list_off[g]:T.list_off[g + 1]]))
        assert diff <= max(1, T.n_groups // 1000), diff
    # every list covers all mass exactly once
    mj = np.concatenate([m[ids], nodes["m"]])
    sums = np.add.reduceat(mj[idx], off[:-1])
    np.testing.assert_allclose(sums, 1.0, rtol=1e-12)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_device_rebuild_run_matches_host_rebuild_run(hh, orc, prec):
    # the whole tree loop with device rebuilds against the same loop with host
    # rebuilds: identical step counts and energies within roundoff
    n = 2048
    x, v, m = synth.plummer(n, 42)
    eps2 = 1e-6
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    out = {}
    for dev in (False, True):
        cfg = hh.hh_config_default()
        cfg.eps2, cfg.precision, cfg.n_crit = eps2, P, 64
        with hh.Context(cfg, n, 2 * n, 4000 * n // 8, n) as ctx:
            ctx.hh_load_particles(x.T, v.T, m)
            ctx.hh_set_rebuild_device(dev)
            ctx.hh_run(0.0, 3 / 64)
            st = ctx.hh_get_state()
            ids = ctx.hh_get_ids()
            c = ctx.hh_get_counters()
        xx = np.zeros((n, 3))
        vv = np.zeros((n, 3))
        xx[ids] = st["x"].T
        vv[ids] = st["v"].T
        out[dev] = (orc.energy(xx, vv, m, eps2), c, xx)
    E0 = orc.energy(x, v, m, eps2)
    assert out[True][1]["rebuilds"] == out[False][1]["rebuilds"] == 4
    assert abs(out[True][1]["particle_steps"] / out[False][1]["particle_steps"] - 1) < 0.01
    assert abs(out[True][0] - out[False][0]) / abs(E0) < 1e-8
    assert np.abs(out[True][2] - out[False][2]).max() < 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_hilbert_order_run_matches_morton_run(hh, orc, prec):
    # Peano-Hilbert order (Section 2) changes where particles and nodes sit,
    # not the tree or the interactions: a run in either order takes the same
    # block steps and reaches the same state within roundoff
    n = 3000
    x, v, m = synth.plummer(n, 44)
    eps2 = 1e-6
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    out = {}
    for order in (hh.HH_ORDER_MORTON, hh.HH_ORDER_HILBERT):
        cfg = hh.hh_config_default()
        cfg.eps2, cfg.precision, cfg.n_crit, cfg.order = eps2, P, 64, order
        with hh.Context(cfg, n, 2 * n, 600 * n, n) as ctx:
            ctx.hh_load_particles(x.T, v.T, m)
            ctx.hh_set_rebuild_device(True)
            ctx.hh_run(0.0, 2 / 64)
            st = ctx.hh_get_state()
            ids = ctx.hh_get_ids()
            c = ctx.hh_get_counters()
        xx = np.zeros((n, 3))
        xx[ids] = st["x"].T
        out[order] = (xx, c)
    (xm, cm), (xh, ch) = out[hh.HH_ORDER_MORTON], out[hh.HH_ORDER_HILBERT]
    if prec == "fp64":
        assert cm["interactions"] == ch["interactions"]
        assert np.abs(xh - xm).max() < 1e-6
    else:
        # FP32 pairwise sums in another order move a few particles across a
        # block-step level boundary; the runs stay within the mixed form's error
        assert abs(ch["interactions"] / cm["interactions"] - 1) < 0.01
        assert np.abs(xh - xm).max() < 1e-4
    assert abs(ch["particle_steps"] / cm["particle_steps"] - 1) < 0.01


def test_device_rebuild_grows_the_list_buffer(hh, orc):
    # list_max far below the need: the device rebuild grows the buffer (and
    # the context's byte count) instead of failing, and the lists are right
    n = 4000
    x, v, m = synth.plummer(n, 45)
    cfg = hh.hh_config_default()
    cfg.n_crit = 64
    z = np.zeros_like(x)
    T = orc.tree_build(x, v, z, z, m, leaf=8, n_crit=64, theta=0.5)
    with hh.Context(cfg, n, 2 * n + 64, 1024, n // 4 + 64) as ctx:
        ctx.hh_load_particles(x.T, v.T, m)
        ctx.hh_set_rebuild_device(True)
        b0 = ctx.device_bytes
        ctx.hh_rebuild(0.0)
        off, idx, gof = ctx.hh_get_lists()
        assert ctx.device_bytes >= b0 + 4 * (len(T.list_idx) - 1024)
        assert np.array_equal(off, T.list_off) and np.array_equal(idx, T.list_idx)
        ctx.hh_run(0.0, 1 / 64)  # the loop runs on the grown lists
        assert ctx.hh_get_counters()["rebuilds"] >= 3


@pytest.mark.parametrize("loop", ["graph", "batch"])
def test_tile_step_counter(hh, loop):
    # every active tile of every block step is counted once: particle steps
    # lie between the tile steps and tile_i times the tile steps
    n = 3000
    x, v, m = synth.plummer(n, 46)
    cfg = hh.hh_config_default()
    cfg.eps2, cfg.n_crit, cfg.tile_i = 1e-6, 64, 16
    with hh.Context(cfg, n, 2 * n, 600 * n, n) as ctx:
        ctx.hh_load_particles(x.T, v.T, m)
        ctx.hh_run(0.0, 0.0)
        ctx.hh_reset_counters()
        if loop == "graph":
            ctx.hh_advance(1 / 64)
        else:
            with hh.Batch(hh.HH_FP64, max_sims=1, max_steps=4096) as b:
                b.hh_batch_run([ctx], [1 / 64])
        c = ctx.hh_get_counters()
        h = ctx.hh_get_tile_histogram()
    assert 0 < c["tile_steps"] <= c["particle_steps"] <= 16 * c["tile_steps"]
    # each corrected particle sits in exactly one evaluated tile of its step
    assert h.sum() == c["tile_steps"] and not h[16:].any()
    assert int((np.arange(1, 33) * h).sum()) == c["particle_steps"]


def test_perfmodel_measures_on_the_gpu(hh):
    from paper_1602_02832_gb300 import perfmodel
    r = perfmodel.measure(4096, 0.5, 64, hh.HH_MIXED, intervals=1, warm=1)
    assert r["particle_steps"] > 0 and r["block_steps"] > 0
    assert 100 < r["N_int"] < 4096 and 1.0 <= r["n_i"] <= 32.0
    assert all(r[k] > 0 for k in ("T_force", "T_predict", "T_tree"))
    rows = perfmodel.sweep_n_i(4096, 0.5, 256, hh.HH_FP64, ks=(1, 3, 8), reps=2)
    assert [q["k"] for q in rows] == [1, 3, 8] and all(q["interactions_per_s"] > 0 for q in rows)


def test_device_rebuild_reports_too_few_cells(hh):
    # room for 10 cells only: the build stops (no cell is written past the
    # capacity and no later level is read) and reports HH_ENOMEM before it
    # reorders anything, so the particle state stays as loaded
    n = 2000
    x, v, m = synth.plummer(n, 47)
    cfg = hh.hh_config_default()
    with hh.Context(cfg, n, n + 10, 600 * n, n) as ctx:
        ctx.hh_load_particles(x.T, v.T, m)
        ctx.hh_set_rebuild_device(True)
        with pytest.raises(hh.HHError) as e:
            ctx.hh_rebuild(0.0)
        assert e.value.code == hh.HH_ENOMEM and "nj_max" in str(e.value)
        with pytest.raises(hh.HHError) as e2:  # no valid lists until a rebuild succeeds
            ctx.hh_step()
        assert e2.value.code == hh.HH_ESTATE
        st = ctx.hh_get_state()  # the state stays readable
        assert np.array_equal(st["x"], np.ascontiguousarray(x.T))
        got = ctx.hh_get_j(0, n)
        assert np.array_equal(got["x"], np.ascontiguousarray(x.T)) and np.array_equal(ctx.hh_get_ids(), np.arange(n))


def test_step_profile_takes_the_same_steps_twice(hh):
    # the per-step profile runs one interval twice from the same state (one
    # launch; one step per launch) and pairs their steps one to one
    import numpy as np
    from paper_1602_02832_gb300 import perfmodel
    rows = perfmodel.step_profile(4096, hh.HH_FP64, {"n_crit": 64, "tile_i": 8, "tile_j": 256}, warm=1)
    A, I, LM, U, P1, P2 = rows.T
    assert len(rows) > 10 and np.all(A >= 1) and np.all(I > 0) and np.all(LM == 0)
    assert np.allclose(U, P1 + P2, rtol=1e-9, atol=1e-3)
    b = perfmodel.step_bins(rows)
    assert sum(x["steps"] for x in b) == len(rows)


def test_device_tree_deeper_than_the_last_one(hh, orc):
    # the level loop first runs to two levels below the last tree's depth and
    # finishes the deeper levels after reading the counts: a shallow tree (a
    # uniform cube) followed by a deep one (a Plummer sphere) takes that path,
    # and the deep tree still equals the oracle's
    n = 20000
    rng = np.random.default_rng(5)
    xu = rng.uniform(-1.0, 1.0, size=(n, 3))
    x, v, m = synth.plummer(n, 43)
    z = np.zeros_like(x)
    Tu = orc.tree_build(xu, v, z, z, m, leaf=8, n_crit=64, theta=0.5)
    T = orc.tree_build(x, v, z, z, m, leaf=8, n_crit=64, theta=0.5)
    cfg = hh.hh_config_default()
    cfg.theta, cfg.n_crit = 0.5, 64
    cells = max(Tu.n_cells, T.n_cells)
    with hh.Context(cfg, n, n + 2 * cells + 64, 2 * max(len(Tu.list_idx), len(T.list_idx)) + 1024,
                    2 * max(Tu.n_groups, T.n_groups) + 64) as ctx:
        ctx.hh_set_rebuild_device(True)
        ctx.hh_load_particles(xu.T, v.T, m)
        ctx.hh_rebuild(0.0)
        assert np.array_equal(ctx.hh_get_ids(), Tu.perm)
        ctx.hh_load_particles(x.T, v.T, m)
        ctx.hh_rebuild(0.0)
        ids = ctx.hh_get_ids()
        off, idx, gof = ctx.hh_get_lists()
        nodes = ctx.hh_get_j(n, ctx.nj - n)
    assert np.array_equal(ids, T.perm) and np.array_equal(gof, T.group_of)
    assert len(nodes["m"]) == T.n_cells
    # node masses summed in another order: within n eps (2e4 terms of 5e-5)
    np.testing.assert_allclose(nodes["m"], T.node_m, rtol=n * 2.3e-16)
    diff = sum(1 for g in range(T.n_groups)
               if not np.array_equal(idx[off[g]:off[g + 1]], T.list_idx[T.list_off[g]:T.list_off[g + 1]]))
    assert diff <= max(1, T.n_groups // 1000), diff
