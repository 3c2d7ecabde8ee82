"""The benchmarked paths, end to end, against the oracle's run (GPU).

The bench times the persistent batched loop (hh_batch_run: k_batch) with the
tree, groups and lists rebuilt on the device every dt_tree, and the server
drives the same loop.  These tests run exactly that path from the same seeded
initial conditions as the FP64 oracle's tree loop (Section 2, steps 1-7) and
compare final states:
- FP64 form: positions and velocities within 1e-6 of the oracle's after
  several rebuild intervals (both integrate the same equations in FP64 with
  the same lists; only summation order differs), equal rebuild counts,
  particle steps within 5%, and energy drift within 2x the oracle's;
- mixed form: energy drift within 2x the oracle's (the stated bar), particle
  steps within 5%, positions within 1e-5.
Energy is kinetic plus half the direct-sum potential (Section 3).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

DTT = 2.0 ** -6
DRIFT_FLOOR = 1e-9  # roundoff of E itself (sum of N terms at 2^-53)


@pytest.fixture(scope="module")
def hh():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1602_02832_gb300 as hh
    return hh


def _cfg(hh, prec, eps2, theta, n_crit):
    c = hh.hh_config_default()
    c.eps2, c.precision, c.theta, c.n_crit = eps2, prec, theta, n_crit
    return c


def _context(hh, prec, x, v, m, eps2, theta, n_crit):
    n = len(m)
    z = np.zeros((3, n))
    T0 = hh.hh_tree_build(x.T, v.T, z, z, m, leaf=8, n_crit=n_crit, theta=theta)
    ctx = hh.Context(_cfg(hh, prec, eps2, theta, n_crit), n, 2 * n + 64, 2 * len(T0.idx) + 4096,
                     2 * T0.n_groups + 64)
    ctx.hh_load_particles(x.T, v.T, m)
    ctx.hh_set_rebuild_device(True)
    ctx.hh_run(0.0, 0.0)  # device rebuild, initial forces, rebuild with node derivatives, initial steps
    return ctx


def _batched_run(hh, prec, sims, t_end, max_steps=4096):
    """sims: list of (x, v, m, eps2, theta, n_crit).  Advances all of them in
    shared hh_batch_run launches, rebuilding each on the device at every
    multiple of dt_tree, to t_end; returns per simulation (x, v, counters)
    with x, v [n, 3] in input order."""
    ctxs = [_context(hh, prec, *s) for s in sims]
    t_stop = np.full(len(ctxs), DTT)
    done = np.zeros(len(ctxs), bool)
    with hh.Batch(prec, max_sims=len(ctxs), max_steps=max_steps) as b:
        launches = 0
        while not done.all():
            live = [i for i in range(len(ctxs)) if not done[i]]
            _, tn, _ = b.hh_batch_run([ctxs[i] for i in live], t_stop[live])
            for i, t in zip(live, tn):
                if t > t_stop[i]:
                    ctxs[i].hh_rebuild(t_stop[i])
                    if t_stop[i] >= t_end:
                        done[i] = True
                    t_stop[i] += DTT
            launches += 1
            assert launches < 100000
    out = []
    for c, (x, v, m, *_rest) in zip(ctxs, sims):
        st = c.hh_get_state()
        ids = c.hh_get_ids()
        assert np.all(st["t"] == t_end)
        xg, vg = np.zeros((len(m), 3)), np.zeros((len(m), 3))
        xg[ids] = st["x"].T
        vg[ids] = st["v"].T
        out.append((xg, vg, c.hh_get_counters()))
        c.close()
    return out


def _oracle(orc, x, v, m, eps2, theta, n_crit, t_end):
    p = orc.RunParams(eps2=eps2, eta=0.02, theta=theta, n_crit=n_crit, use_tree=True)
    return orc.run(x, v, m, t_end, p)


def _drift(orc, x0, v0, x1, v1, m, eps2):
    E0 = orc.energy(x0, v0, m, eps2)
    return abs(orc.energy(x1, v1, m, eps2) - E0) / abs(E0)


def _compare(orc, fp64, sim, gpu, ref, t_end, label):
    x, v, m, eps2, theta, n_crit = sim
    xg, vg, c = gpu
    dE_g = _drift(orc, x, v, xg, vg, m, eps2)
    dE_o = _drift(orc, x, v, ref["x"], ref["v"], m, eps2)
    dx = np.abs(xg - ref["x"]).max()
    dv = np.abs(vg - ref["v"]).max()
    ps_ratio = c["particle_steps"] / ref["stats"]["particle_steps"]
    print(f"\n{label}: N={len(m)} theta={theta} to t={t_end}: dE/E gpu {dE_g:.3e} oracle {dE_o:.3e}; "
          f"max |dx| {dx:.2e} |dv| {dv:.2e}; particle steps gpu/oracle {ps_ratio:.4f}; "
          f"rebuilds {c['rebuilds']} / {ref['stats']['rebuilds']}")
    assert dE_g <= 2 * dE_o + DRIFT_FLOOR
    assert abs(ps_ratio - 1) < 0.05
    assert c["rebuilds"] == ref["stats"]["rebuilds"]
    if fp64:
        assert dx < 1e-6 and dv < 1e-6
    else:
        assert dx < 1e-5 and dv < 1e-5


SIMS = [(1024, 21, 0.5, False), (2048, 22, 0.3, True), (3000, 23, 0.7, False)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_loop_with_device_rebuilds_matches_oracle(hh, orc, prec):
    # three simulations of different N, theta and mass spectra share every
    # launch of the persistent loop; three rebuild intervals on the device
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    t_end = 3 * DTT
    sims = []
    for n, seed, theta, sal in SIMS:
        x, v, m = (synth.plummer_salpeter if sal else synth.plummer)(n, seed)
        sims.append((x, v, m, 1e-6, theta, 32))
    gpu = _batched_run(hh, P, sims, t_end)
    for s, g in zip(sims, gpu):
        ref = _oracle(orc, *s, t_end)
        _compare(orc, P == hh.HH_FP64, s, g, ref, t_end, f"batched {prec}")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_served_requests_match_oracle(hh, orc, prec):
    # the continuous-batching server (device rebuilds, launches of 16 global
    # steps, requests of different end times sharing launches) against the
    # oracle run of each request alone
    from paper_1602_02832_gb300 import serve
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    specs = [(1500, 31, 2 * DTT, True), (700, 32, DTT, False), (2500, 33, 3 * DTT, False)]
    reqs = []
    for rid, (n, seed, t_end, sal) in enumerate(specs):
        x, v, m = (synth.plummer_salpeter if sal else synth.plummer)(n, seed)
        reqs.append(serve.SimRequest(rid, x, v, m, t_end, arrival_s=0.0))
    srv = serve.Server(precision=P, budget_bytes=10 ** 11, max_sims=4, max_steps=16, eps2=1e-6, n_crit=32,
                       rebuild_device=True)
    res, _ = srv.run(reqs, realtime=False)
    srv.close()
    assert sorted(r.rid for r in res) == [0, 1, 2]
    for r in res:
        q = reqs[r.rid]
        ref = _oracle(orc, q.x, q.v, q.m, 1e-6, 0.5, 32, q.t_end)
        dE_g = _drift(orc, q.x, q.v, r.x, r.v, q.m, 1e-6)
        dE_o = _drift(orc, q.x, q.v, ref["x"], ref["v"], q.m, 1e-6)
        dx = np.abs(r.x - ref["x"]).max()
        dv = np.abs(r.v - ref["v"]).max()
        ps = r.particle_steps / ref["stats"]["particle_steps"]
        print(f"\nserved {prec} request {r.rid} (N={len(q.m)}, t_end={q.t_end}): dE/E {dE_g:.3e} oracle "
              f"{dE_o:.3e}; max |dx| {dx:.2e} |dv| {dv:.2e}; particle steps ratio {ps:.4f}")
        assert dE_g <= 2 * dE_o + DRIFT_FLOOR
        assert abs(ps - 1) < 0.05
        lim = 1e-6 if P == hh.HH_FP64 else 1e-5
        assert dx < lim and dv < lim


@pytest.fixture(scope="module")
def big_oracle(orc):
    """The oracle's run of the N = 32768 Plummer sphere (theta 0.5, n_crit 64,
    eps = 1e-4) over three rebuild intervals, shared by both forms."""
    n = 32768
    x, v, m = synth.plummer(n, 0)
    sim = (x, v, m, 1e-8, 0.5, 64)
    return sim, _oracle(orc, *sim, 3 * DTT)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_energy_drift_n32768_batched_vs_oracle(hh, orc, big_oracle, prec):
    # the full run's settings (eta 0.02, dt in [2^-30, 2^-6], dt_tree 1/64,
    # theta 0.5, eps 1e-4) at half its N, three intervals, device rebuilds
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    sim, ref = big_oracle
    gpu = _batched_run(hh, P, [sim], 3 * DTT)[0]
    _compare(orc, P == hh.HH_FP64, sim, gpu, ref, 3 * DTT, f"N=32768 {prec}")
