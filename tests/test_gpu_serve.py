"""Continuous-batching server on the GPU: every simulation's result is the same
alone and in the mix (bitwise: its tiles, active sets and list parts are its
own and its sums run in fixed order), also when a small memory budget makes
requests queue, with host rebuilds and with the server's automatic choice
(device builds, batched when several simulations reach their rebuild time in
one launch, single when one does)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1602_02832_gb300 as hh
    from paper_1602_02832_gb300 import serve
    return hh, serve


def _requests(serve):
    specs = [(400, 11, 1 / 64, False), (1200, 12, 2 / 64, True), (256, 13, 2 / 64, False), (900, 14, 1 / 64, True)]
    out = []
    for rid, (n, seed, t_end, sal) in enumerate(specs):
        x, v, m = (synth.plummer_salpeter if sal else synth.plummer)(n, seed)
        out.append(serve.SimRequest(rid, x, v, m, t_end, arrival_s=0.0))
    return out


@pytest.mark.parametrize("prec,rebuild", [("mixed", False), ("fp64", False), ("mixed", "auto"), ("fp64", "auto")])
def test_same_alone_and_in_the_mix(env, prec, rebuild):
    hh, serve = env
    P = hh.HH_MIXED if prec == "mixed" else hh.HH_FP64
    reqs = _requests(serve)
    alone = {}
    kw = dict(precision=P, max_sims=4, max_steps=16, eps2=1e-6, n_crit=32, rebuild_device=rebuild)
    for r in reqs:
        srv = serve.Server(budget_bytes=10 ** 11, **kw)
        res, _ = srv.run([r], realtime=False)
        srv.close()
        alone[r.rid] = res[0]
    for budget in (10 ** 11, None):
        if budget is None:  # room for about two of the simulations at a time
            srv0 = serve.Server(**kw)
            est = sorted(srv0.estimate_bytes(r)[0] for r in reqs)
            srv0.close()
            budget = est[-1] + est[-2]
        srv = serve.Server(budget_bytes=budget, **kw)
        res, stats = srv.run(reqs, realtime=False)
        srv.close()
        assert sorted(r.rid for r in res) == [0, 1, 2, 3]
        for r in res:
            a = alone[r.rid]
            assert np.array_equal(r.x, a.x) and np.array_equal(r.v, a.v)
            assert r.block_steps == a.block_steps and r.interactions == a.interactions
        assert stats.launches > 0 and len(stats.step_us) > 0
