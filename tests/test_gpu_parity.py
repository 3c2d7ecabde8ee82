"""GPU parity: libhh's CUDA path against the FP64 oracle, element by element.

Every comparison feeds both sides the same seeded inputs and the same
interaction lists (built by the oracle), so the only differences are rounding
order (FP64 form) or the mixed-precision arithmetic (HH_MIXED).

Tolerances (tests/_parity.py), for every particle, no quantiles.  FP64 form:
1e-11 relative covers the reordered summation of up to ~1e4 terms (n * 2^-53
* cancellation).  Mixed form: acceleration and potential <= 1e-6, jerk <= 1e-5
relative (the stated bars); where a particle's jerk nearly cancels, its error
may instead be <= 1e-6 of J_scale = sum_j m_j (|w| s^-3/2 + 3 |r.w| |r| s^-5/2),
the size of the terms it sums.
"""
import numpy as np
import pytest

import _parity
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hh():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1602_02832_gb300 as hh
    return hh


def _cfg(hh, prec, eps2=1e-8, **kw):
    c = hh.hh_config_default()
    c.eps2 = eps2
    c.precision = prec
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _ctx_from_tree(hh, cfg, T, xj, vj, aj, jj, mj, tj):
    n = T.n
    nj = len(mj)
    ctx = hh.Context(cfg, n, nj, max(1, len(T.list_idx)), T.n_groups)
    ctx.hh_set_j(0, xj.T, vj.T, aj.T, jj.T, mj, tj)
    ctx.hh_set_lists(n, nj, T.list_off, T.list_idx, T.group_of)
    return ctx


def _setup_plummer(orc, n, seed, theta, n_crit, salpeter=False, eps2=1e-8, t_spread=False):
    x, v, m = (synth.plummer_salpeter if salpeter else synth.plummer)(n, seed)
    a, j, _ = orc.direct_force(x, v, m, eps2)
    T = orc.tree_build(x, v, a, j, m, leaf=8, n_crit=n_crit, theta=theta)
    xj, vj, aj, jj, mj = T.j_array(x, v, a, j, m)
    tj = np.zeros(len(mj))
    if t_spread:
        # particles at assorted earlier block times, nodes at the tree time 0
        rng = np.random.default_rng(seed)
        tj[:n] = rng.integers(0, 8, size=n) * 2.0 ** -9
    return x, v, m, T, xj, vj, aj, jj, mj, tj


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("theta,n_crit,salp", [(0.5, 64, False), (0.3, 200, True), (0.75, 16, False)])
def test_list_force_parity_n4096(hh, orc, prec, theta, n_crit, salp):
    # The small configuration: N = 4096 Plummer, eps = 1e-4, one force
    # evaluation of all particles from Barnes-Hut lists (leaf 8).
    x, v, m, T, xj, vj, aj, jj, mj, tj = _setup_plummer(orc, 4096, 0, theta, n_crit, salp)
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    with _ctx_from_tree(hh, _cfg(hh, P), T, xj, vj, aj, jj, mj, tj) as ctx:
        ctx.hh_predict(0.0)
        ia = np.arange(4096, dtype=np.int32)
        acc, jerk, pot = ctx.hh_force(ia)
    ra, rj, rp = orc.list_force(xj, vj, mj, ia, T.group_of, T.list_off, T.list_idx, 1e-8)
    _parity.check(P == hh.HH_FP64, acc, jerk, pot, ra, rj, rp,
                  lambda k: _parity.jscale(xj, vj, mj, T.group_of[ia[k]], T.list_off, T.list_idx, ia[k], 1e-8),
                  f"{prec} theta={theta} n_crit={n_crit}")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_predict_and_force_parity_with_time_offsets(hh, orc, prec):
    # Particles sit at different earlier block times and the nodes at the
    # tree time; hh_predict moves every j entry to t = 2^-6 before the force.
    x, v, m, T, xj, vj, aj, jj, mj, tj = _setup_plummer(orc, 3000, 1, 0.5, 48, t_spread=True)
    t = 2.0 ** -6
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    with _ctx_from_tree(hh, _cfg(hh, P), T, xj, vj, aj, jj, mj, tj) as ctx:
        ctx.hh_predict(t)
        ia = np.arange(0, 3000, 3, dtype=np.int32)
        acc, jerk, pot = ctx.hh_force(ia)
    xp, vp = orc.predict(xj, vj, aj, jj, tj, t)
    ra, rj, rp = orc.list_force(xp, vp, mj, ia, T.group_of[ia], T.list_off, T.list_idx, 1e-8)
    _parity.check(P == hh.HH_FP64, acc, jerk, pot, ra, rj, rp,
                  lambda k: _parity.jscale(xp, vp, mj, T.group_of[ia[k]], T.list_off, T.list_idx, ia[k], 1e-8),
                  f"{prec} predicted to 2^-6")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_theta_zero_equals_direct_sum(hh, orc, prec):
    # theta = 0: every list is all particles, so the GPU list force is the
    # direct N^2 sum of the original Hermite loop.
    n = 1000
    x, v, m = synth.plummer(n, 2)
    eps2 = 1e-6
    a, j, _ = orc.direct_force(x, v, m, eps2)
    T = orc.tree_build(x, v, a, j, m, leaf=8, n_crit=40, theta=0.0)
    xj, vj, aj, jj, mj = T.j_array(x, v, a, j, m)
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    with _ctx_from_tree(hh, _cfg(hh, P, eps2), T, xj, vj, aj, jj, mj, np.zeros(len(mj))) as ctx:
        ctx.hh_predict(0.0)
        acc, jerk, pot = ctx.hh_force(np.arange(n, dtype=np.int32))
    ia = np.arange(n, dtype=np.int32)
    _parity.check(P == hh.HH_FP64, acc, jerk, pot, a[T.perm], j[T.perm],
                  orc.direct_force(x, v, m, eps2)[2][T.perm],
                  lambda k: _parity.jscale(xj, vj, mj, T.group_of[ia[k]], T.list_off, T.list_idx, ia[k], eps2),
                  f"{prec} theta=0 vs direct sum")


@pytest.mark.parametrize("tile_i,tile_j", [(1, 512), (5, 256), (32, 512), (32, 4096)])
def test_ragged_tiles_and_sparse_active_sets(hh, orc, tile_i, tile_j):
    # Static i tiles of 1, 5 or 32 particles; active sets of assorted sizes and
    # gaps (including single particles and whole groups).
    x, v, m, T, xj, vj, aj, jj, mj, tj = _setup_plummer(orc, 2000, 3, 0.5, 70)
    rng = np.random.default_rng(4)
    ref = orc.list_force(xj, vj, mj, np.arange(2000), T.group_of, T.list_off, T.list_idx, 1e-8)
    # tile_j = list entries per part: 256 splits every list into many parts
    # (partials reduced by the last arriving CTA), 4096 keeps most whole
    with _ctx_from_tree(hh, _cfg(hh, hh.HH_MIXED, tile_i=tile_i, tile_j=tile_j), T, xj, vj, aj, jj, mj, tj) as ctx:
        ctx.hh_predict(0.0)
        for frac in (0.001, 0.05, 0.3, 1.0):
            ia = np.sort(rng.choice(2000, size=max(1, int(frac * 2000)), replace=False)).astype(np.int32)
            acc, jerk, pot = ctx.hh_force(ia)
            _parity.check(False, acc, jerk, pot, ref[0][ia], ref[1][ia], ref[2][ia],
                          lambda k, ia=ia: _parity.jscale(xj, vj, mj, T.group_of[ia[k]], T.list_off, T.list_idx,
                                                          ia[k], 1e-8),
                          f"mixed tile_i={tile_i} tile_j={tile_j} active {len(ia)}")
        # an empty active set is a no-op
        acc, jerk, pot = ctx.hh_force(np.zeros(0, np.int32))
        assert acc.shape == (3, 0)


def test_results_independent_of_co_active_particles(hh, orc):
    # A particle's result must not depend on which other particles are active
    # beyond its tile's active count: same (particle, tile count) -> bitwise
    # equal; any count -> within the FP64 reordering bound.
    x, v, m, T, xj, vj, aj, jj, mj, tj = _setup_plummer(orc, 1500, 5, 0.5, 64)
    with _ctx_from_tree(hh, _cfg(hh, hh.HH_FP64), T, xj, vj, aj, jj, mj, tj) as ctx:
        ctx.hh_predict(0.0)
        full = ctx.hh_force(np.arange(1500, dtype=np.int32))
        again = ctx.hh_force(np.arange(1500, dtype=np.int32))
        for q in range(3):
            assert np.array_equal(full[q], again[q])
        one = ctx.hh_force(np.array([777], np.int32))
        assert np.allclose(one[0][:, 0], full[0][:, 777], rtol=1e-13, atol=0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_large_sampled_parity_n65536(hh, orc, prec):
    # N = 65536 (the full-run size): lists from the library's host builder,
    # all particles on the GPU, the oracle on a sample of 400 particles.
    n = 65536
    x, v, m = synth.plummer(n, 0)
    eps2 = 1e-8
    z = np.zeros((3, n))
    Tp = hh.hh_tree_build(x.T, v.T, z, z, m, leaf=8, n_crit=64, theta=0.5)
    nj = n + Tp.n_nodes
    xj = np.concatenate([x[Tp.perm], Tp.node_x.T])
    vj = np.concatenate([v[Tp.perm], Tp.node_v.T])
    zj = np.zeros_like(xj)
    mj = np.concatenate([m[Tp.perm], Tp.node_m])
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    cfg = _cfg(hh, P, eps2)
    with hh.Context(cfg, n, nj, len(Tp.idx), Tp.n_groups) as ctx:
        ctx.hh_set_j(0, xj.T, vj.T, zj.T, zj.T, mj, np.zeros(nj))
        ctx.hh_set_lists(n, nj, Tp.off, Tp.idx, Tp.group_of)
        ctx.hh_predict(0.0)
        acc, jerk, pot = ctx.hh_force(np.arange(n, dtype=np.int32))
    s = np.random.default_rng(0).choice(n, 400, replace=False).astype(np.int32)
    ra, rj, rp = orc.list_force(xj, vj, mj, s, Tp.group_of[s], Tp.off, Tp.idx, eps2)
    _parity.check(P == hh.HH_FP64, acc[:, s], jerk[:, s], pot[s], ra, rj, rp,
                  lambda k: _parity.jscale(xj, vj, mj, Tp.group_of[s[k]], Tp.off, Tp.idx, s[k], eps2),
                  f"{prec} N=65536, 400 sampled particles")
    assert np.all(np.isfinite(acc)) and np.all(np.isfinite(jerk)) and np.all(np.isfinite(pot))


def test_large_sampled_parity_n1m_salpeter_mixed(hh, orc):
    # N = 10^6 Plummer with a Salpeter spectrum (slope -2.35, mass ratio 100),
    # mixed form; oracle on 200 sampled particles of the same lists.
    n = 1 << 20
    x, v, m = synth.plummer_salpeter(n, 0)
    eps2 = 1e-8
    z = np.zeros((3, n))
    Tp = hh.hh_tree_build(x.T, v.T, z, z, m, leaf=8, n_crit=128, theta=0.5)
    nj = n + Tp.n_nodes
    xj = np.concatenate([x[Tp.perm], Tp.node_x.T])
    vj = np.concatenate([v[Tp.perm], Tp.node_v.T])
    zj = np.zeros_like(xj)
    mj = np.concatenate([m[Tp.perm], Tp.node_m])
    with hh.Context(_cfg(hh, hh.HH_MIXED, eps2), n, nj, len(Tp.idx), Tp.n_groups) as ctx:
        ctx.hh_set_j(0, xj.T, vj.T, zj.T, zj.T, mj, np.zeros(nj))
        ctx.hh_set_lists(n, nj, Tp.off, Tp.idx, Tp.group_of)
        ctx.hh_predict(0.0)
        s = np.random.default_rng(1).choice(n, 200, replace=False).astype(np.int32)
        acc, jerk, pot = ctx.hh_force(s)
    ra, rj, rp = orc.list_force(xj, vj, mj, s, Tp.group_of[s], Tp.off, Tp.idx, eps2)
    _parity.check(False, acc, jerk, pot, ra, rj, rp,
                  lambda k: _parity.jscale(xj, vj, mj, Tp.group_of[s[k]], Tp.off, Tp.idx, s[k], eps2),
                  "mixed N=2^20 Salpeter, 200 sampled particles")


def test_corrector_and_block_step_parity(hh, orc):
    # One explicit corrector pass: GPU hh_correct against the oracle's
    # corrector, Aarseth criterion and block quantisation, particle by particle.
    n = 1200
    eps2 = 1e-6
    x, v, m = synth.plummer(n, 6)
    a0, j0, _ = orc.direct_force(x, v, m, eps2)
    T = orc.tree_build(x, v, a0, j0, m, leaf=8, n_crit=64, theta=0.0)  # direct lists
    xj, vj, aj, jj, mj = T.j_array(x, v, a0, j0, m)
    tj = np.zeros(len(mj))
    dt = np.array([orc.initial_dt(0.01, aj[k], jj[k], 2.0 ** -30, 2.0 ** -6) for k in range(n)])
    t_next = dt.min()
    act = np.nonzero(dt == t_next)[0].astype(np.int32)
    assert 0 < len(act) < n
    with _ctx_from_tree(hh, _cfg(hh, hh.HH_FP64, eps2), T, xj, vj, aj, jj, mj, tj) as ctx:
        ctx.hh_set_dt(dt)
        ctx.hh_predict(t_next)
        acc, jerk, pot = ctx.hh_force(act)
        ctx.hh_correct(t_next, act)
        st = ctx.hh_get_state()
        # a particle that is not due is rejected by the device check
        late = np.array([np.nonzero(dt > t_next)[0][0]], np.int32)
        ctx.hh_predict(t_next)
        ctx.hh_force(late)
        with pytest.raises(hh.HHError):
            ctx.hh_correct(t_next, late)
    xp, vp = orc.predict(xj, vj, aj, jj, tj, t_next)
    ra, rj, _ = orc.list_force(xp, vp, mj, act, T.group_of[act], T.list_off, T.list_idx, eps2)
    mism = 0
    for k, i in enumerate(act):
        x1, v1, a2e, a3 = orc.correct_one(t_next, xp[i], vp[i], aj[i], jj[i], ra[k], rj[k])
        np.testing.assert_allclose(st["x"][:, i], x1, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(st["v"][:, i], v1, rtol=1e-12, atol=1e-14)
        want = orc.aarseth_dt(0.02, ra[k], rj[k], a2e, a3)
        nd = orc.block_dt(want, dt[i], t_next, 2.0 ** -30, 2.0 ** -6)
        if st["dt"][i] != nd:
            # only a request within rounding of a power-of-two boundary may differ
            mism += 1
            assert abs(np.log2(want) - np.round(np.log2(want))) < 1e-9
        assert st["t"][i] == t_next
    assert mism <= 1
    others = np.setdiff1d(np.arange(n), act)
    assert np.array_equal(st["x"][:, others], xj[others].T)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_device_block_step_matches_oracle_step(hh, orc, prec):
    # hh_step: block selection, prediction, force and correction on the device
    # against the same block step done by the oracle's functions.
    n = 800
    eps2 = 1e-6
    x, v, m = synth.plummer(n, 7)
    a0, j0, _ = orc.direct_force(x, v, m, eps2)
    T = orc.tree_build(x, v, a0, j0, m, leaf=8, n_crit=32, theta=0.5)
    xj, vj, aj, jj, mj = T.j_array(x, v, a0, j0, m)
    tj = np.zeros(len(mj))
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    with _ctx_from_tree(hh, _cfg(hh, P, eps2), T, xj, vj, aj, jj, mj, tj) as ctx:
        ctx.hh_init_dt()
        dt0 = ctx.hh_get_state()["dt"]
        t1, na = ctx.hh_step()
        st = ctx.hh_get_state()
        c = ctx.hh_get_counters()
    dt_ref = np.array([orc.initial_dt(0.01, aj[k], jj[k], 2.0 ** -30, 2.0 ** -6) for k in range(n)])
    assert np.array_equal(dt0, dt_ref)
    assert t1 == dt_ref.min()
    act = np.nonzero(dt_ref == t1)[0]
    assert na == len(act)
    assert c["particle_steps"] == na and c["block_steps"] == 1
    assert c["interactions"] == sum(T.list_off[g + 1] - T.list_off[g] - 1 for g in T.group_of[act])
    xp, vp = orc.predict(xj, vj, aj, jj, tj, t1)
    ra, rj, _ = orc.list_force(xp, vp, mj, act.astype(np.int32), T.group_of[act], T.list_off, T.list_idx, eps2)
    tol = 1e-12 if P == hh.HH_FP64 else 1e-9
    for k, i in enumerate(act):
        x1, v1, _, _ = orc.correct_one(t1, xp[i], vp[i], aj[i], jj[i], ra[k], rj[k])
        np.testing.assert_allclose(st["x"][:, i], x1, rtol=tol, atol=1e-14)
        assert st["t"][i] == t1


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_run_energy_vs_oracle(hh, orc, prec):
    # The whole tree loop on the device (rebuild every dt_tree on the host with
    # the library's builder) against the oracle's run: same step counts within
    # a few percent and energy drift within 2x the oracle's (+ roundoff floor).
    n = 512
    x, v, m = synth.plummer(n, 8)
    eps2 = 1e-4
    t_end = 0.125
    p = orc.RunParams(eps2=eps2, eta=0.02, theta=0.5, n_crit=32, use_tree=True)
    r = orc.run(x, v, m, t_end, p)
    E0 = orc.energy(x, v, m, eps2)
    dE_orc = abs(orc.energy(r["x"], r["v"], m, eps2) - E0) / abs(E0)
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    cfg = _cfg(hh, P, eps2, n_crit=32, theta=0.5)
    with hh.Context(cfg, n, 4 * n, 64 * n * n // 32, n) as ctx:
        ctx.hh_load_particles(x.T, v.T, m)
        ctx.hh_run(0.0, t_end)
        st = ctx.hh_get_state()
        ids = ctx.hh_get_ids()
        c = ctx.hh_get_counters()
    xg = np.zeros((n, 3))
    vg = np.zeros((n, 3))
    xg[ids] = st["x"].T
    vg[ids] = st["v"].T
    assert np.all(st["t"] == t_end)
    dE_gpu = abs(orc.energy(xg, vg, m, eps2) - E0) / abs(E0)
    print(f"\n{prec}: dE/E gpu {dE_gpu:.3e} oracle {dE_orc:.3e}; steps gpu {c['particle_steps']} "
          f"oracle {r['stats']['particle_steps']}")
    assert dE_gpu <= 2 * dE_orc + 1e-9
    assert abs(c["particle_steps"] / r["stats"]["particle_steps"] - 1) < 0.05
    assert c["rebuilds"] == r["stats"]["rebuilds"]
    if P == hh.HH_FP64:
        assert np.abs(xg - r["x"]).max() < 1e-6


def test_input_validation_errors(hh, orc):
    x, v, m, T, xj, vj, aj, jj, mj, tj = _setup_plummer(orc, 300, 9, 0.5, 32)
    nj = len(mj)
    with _ctx_from_tree(hh, _cfg(hh, hh.HH_FP64), T, xj, vj, aj, jj, mj, tj) as ctx:
        bad = T.list_idx.copy()
        bad[5] = nj + 3
        with pytest.raises(hh.HHError) as e:
            ctx.hh_set_lists(300, nj, T.list_off, bad, T.group_of)
        assert e.value.code == hh.HH_EINVAL
        with pytest.raises(hh.HHError):
            ctx.hh_force(np.array([1, 2], np.int32))  # no predict since lists were (re)set
        ctx.hh_set_lists(300, nj, T.list_off, T.list_idx, T.group_of)
        ctx.hh_predict(0.0)
        with pytest.raises(hh.HHError):
            ctx.hh_force(np.array([3, 3], np.int32))
        with pytest.raises(hh.HHError):
            ctx.hh_force(np.array([300], np.int32))
        mm = mj.copy()
        mm[0] = -1.0
        with pytest.raises(hh.HHError):
            ctx.hh_set_j(0, xj.T, vj.T, aj.T, jj.T, mm, tj)
        # still usable after the errors
        ctx.hh_set_j(0, xj.T, vj.T, aj.T, jj.T, mj, tj)
        ctx.hh_predict(0.0)
        acc, _, _ = ctx.hh_force(np.arange(300, dtype=np.int32))
        assert np.all(np.isfinite(acc))
