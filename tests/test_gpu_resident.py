"""The batch's resident set through the C ABI (GPU): admission by device-memory
budget and free slots, one launch per hh_batch_step with the due rebuilds,
each finished simulation reported once, retirement freeing its budget share,
and a particle cap per launch.  Every simulation's final state must equal,
bit for bit, the state it reaches alone through hh_batch_run with the same
rebuilds (its tiles, active sets and list parts are its own; sums run in
fixed order)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

DTT = 2.0 ** -6
SPECS = [(500, 41, False, 2 * DTT), (800, 42, True, DTT), (1200, 43, False, 2 * DTT)]


@pytest.fixture(scope="module")
def hh():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1602_02832_gb300 as hh
    return hh


def _ctx(hh, prec, n, seed, sal):
    x, v, m = (synth.plummer_salpeter if sal else synth.plummer)(n, seed)
    c = hh.hh_config_default()
    c.eps2, c.precision, c.n_crit = 1e-6, prec, 32
    ctx = hh.Context(c, n, 2 * n + 64, 64 * n * max(1, n // 16), n)
    ctx.hh_load_particles(x.T, v.T, m)
    ctx.hh_set_rebuild_device(True)
    ctx.hh_run(0.0, 0.0)
    return ctx


def _by_id(ctx):
    """State arrays indexed by particle id (a rebuild reorders the slots)."""
    st = ctx.hh_get_state()
    ids = ctx.hh_get_ids()
    out = {}
    for k, a in st.items():
        b = np.zeros_like(a)
        b[..., ids] = a
        out[k] = b
    return out


def _alone(hh, prec, n, seed, sal, t_end):
    # the rebuilds hh_batch_step makes: at every interval end before t_end
    with _ctx(hh, prec, n, seed, sal) as c, hh.Batch(prec, max_sims=1, max_steps=64) as b:
        t = 0.0
        while t < t_end:
            while True:
                _, tn, _ = b.hh_batch_run([c], [t + DTT])
                if tn[0] > t + DTT:
                    break
            if t + DTT < t_end:
                c.hh_rebuild(t + DTT)
            t += DTT
        return _by_id(c)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_resident_set_budget_slots_retire_and_results(hh, prec):
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    ref = [_alone(hh, P, n, seed, sal, te) for n, seed, sal, te in SPECS]
    ctxs = [_ctx(hh, P, n, seed, sal) for n, seed, sal, _ in SPECS]
    by_h = {c.h.value: k for k, c in enumerate(ctxs)}
    with hh.Batch(P, max_sims=2, max_steps=64) as b:
        nbytes = [c.device_bytes for c in ctxs]
        # room for 0 + 1 (and for 0 + 2 once 1 retires), not for all three
        assert nbytes[0] < nbytes[1] < nbytes[2]
        b.hh_batch_set_budget(nbytes[1] + nbytes[2])
        assert b.hh_batch_admit(ctxs[0], SPECS[0][3]) and b.hh_batch_admit(ctxs[1], SPECS[1][3])
        assert not b.hh_batch_admit(ctxs[2], SPECS[2][3])  # no slot and no budget left: nothing changes
        assert b.hh_batch_resident() == (2, 2, nbytes[0] + nbytes[1])
        assert b.hh_batch_resident()[2] + nbytes[2] > nbytes[1] + nbytes[2]
        with pytest.raises(hh.HHError):
            b.hh_batch_admit(ctxs[0], 4 * DTT)  # already resident
        done_order, waiting, calls = [], [2], 0
        while len(done_order) < 3:
            steps, launched, done, us = b.hh_batch_step()
            calls += 1
            assert calls < 10000 and b.hh_batch_resident()[0] > 0
            for h in done:
                k = by_h[h]
                assert k not in done_order  # reported once
                done_order.append(k)
                st = ctxs[k].hh_get_state()
                assert np.all(st["t"] == SPECS[k][3])
                b.hh_batch_retire(ctxs[k])
                if waiting and b.hh_batch_admit(ctxs[waiting[0]], SPECS[waiting[0]][3]):
                    waiting.pop(0)
        assert done_order[0] == 1  # the shortest run finishes first
        assert b.hh_batch_resident() == (0, 0, 0)
        with pytest.raises(hh.HHError):
            b.hh_batch_retire(ctxs[0])  # not resident any more
    for c, st in zip(ctxs, ref):
        got = _by_id(c)
        for k in ("x", "v", "a", "jk", "t", "dt"):
            assert np.array_equal(got[k], st[k]), k
        c.close()


def test_resident_set_particle_cap_and_bad_requests(hh):
    P = hh.HH_MIXED
    ref = [_alone(hh, P, n, seed, sal, te) for n, seed, sal, te in SPECS]
    ctxs = [_ctx(hh, P, n, seed, sal) for n, seed, sal, _ in SPECS]
    with hh.Batch(P, max_sims=4, max_steps=64) as b:
        b.hh_batch_set_budget(0, 900)  # no budget limit; at most 900 particles per launch
        with pytest.raises(hh.HHError):
            b.hh_batch_admit(ctxs[0], 0.01)  # not a multiple of dt_tree
        with pytest.raises(hh.HHError):
            b.hh_batch_set_budget(-1, 0)
        for c, s in zip(ctxs, SPECS):
            assert b.hh_batch_admit(c, s[3])
        finished = 0
        for _ in range(10000):
            steps, launched, done, _ = b.hh_batch_step()
            # 500 + 800 > 900 and every simulation alone fits or is alone
            assert launched <= 1
            for h in done:
                b.hh_batch_retire([c for c in ctxs if c.h.value == h][0])
                finished += 1
            if finished == 3:
                break
        assert finished == 3
    for c, st in zip(ctxs, ref):
        got = _by_id(c)
        for k in ("x", "v", "t", "dt"):
            assert np.array_equal(got[k], st[k]), k
        c.close()
