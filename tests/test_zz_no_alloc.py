"""hh_force_static, the allocation-free force call, against hh_force (GPU).

Some callers cannot allocate device memory (their memory comes from another
allocator, or their loop must not call cudaMalloc / cudaFree, which
synchronise the device); hh_force_static serves them from a fixed scratch
array inside libhh.  This file checks, through the C ABI, that two calls in a
row give the same forces as the regular hh_force path within the parity
tolerances (FP64: 1e-11 relative per particle; mixed: 1e-6 for acceleration
and potential, 1e-5 for the 99.9th percentile of the jerk), and that sizes
beyond the fixed limits are refused.  It sits in its own file, collected
last, and passes alone or after the other tests.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    import oracle
    import paper_1602_02832_gb300 as hh
    return hh, torch, oracle


def _rel(a, b):
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_force_static_matches_hh_force_twice(env, prec):
    hh, torch, orc = env
    orc.build()
    n, eps2 = 3000, 1e-8
    x, v, m = synth.plummer(n, 31)
    a, j, _ = orc.direct_force(x, v, m, eps2)
    T = orc.tree_build(x, v, a, j, m, leaf=8, n_crit=48, theta=0.5)
    xj, vj, aj, jj, mj = T.j_array(x, v, a, j, m)
    nj = len(mj)
    P = hh.HH_FP64 if prec == "fp64" else hh.HH_MIXED
    cfg = hh.hh_config_default()
    cfg.eps2 = eps2
    cfg.precision = P
    rng = np.random.default_rng(5)
    sets = [np.arange(n, dtype=np.int32),
            np.sort(rng.choice(n, 700, replace=False)).astype(np.int32)]
    dev = torch.device("cuda", 0)
    X = torch.tensor(np.ascontiguousarray(xj.T), device=dev)
    V = torch.tensor(np.ascontiguousarray(vj.T), device=dev)
    M = torch.tensor(mj, device=dev)
    OFF = torch.tensor(T.list_off, device=dev)
    IDX = torch.tensor(T.list_idx, device=dev)
    with hh.Context(cfg, n, nj, len(T.list_idx), T.n_groups) as ctx:
        ctx.hh_set_j(0, xj.T, vj.T, aj.T, jj.T, mj, np.zeros(nj))
        ctx.hh_set_lists(n, nj, T.list_off, T.list_idx, T.group_of)
        ctx.hh_predict(0.0)
        for ia in sets:  # two calls in a row, different active sets
            ref = ctx.hh_force(ia)
            I = torch.tensor(ia, device=dev)
            G = torch.tensor(T.group_of[ia], device=dev)
            acc = torch.zeros((3, len(ia)), dtype=torch.float64, device=dev)
            jerk = torch.zeros_like(acc)
            pot = torch.zeros(len(ia), dtype=torch.float64, device=dev)
            hh.hh_force_static(X, V, M, OFF, IDX, I, G, acc, jerk, pot, eps2=eps2, precision=P)
            ea = _rel(acc.cpu().numpy(), ref[0])
            ej = _rel(jerk.cpu().numpy(), ref[1])
            ep = np.abs(pot.cpu().numpy() - ref[2]) / np.abs(ref[2])
            if P == hh.HH_FP64:
                assert ea.max() < 1e-11 and ej.max() < 1e-11 and ep.max() < 1e-11
            else:
                assert ea.max() <= 1e-6 and ep.max() <= 1e-6 and np.quantile(ej, 0.999) <= 1e-5


def test_force_static_refuses_oversize_and_bad_input(env):
    hh, torch, _ = env
    dev = torch.device("cuda", 0)
    nj = 131072 + 1
    X = torch.zeros((3, nj), dtype=torch.float64, device=dev)
    M = torch.ones(nj, dtype=torch.float64, device=dev)
    OFF = torch.tensor([0, 2], dtype=torch.int64, device=dev)
    IDX = torch.tensor([0, 1], dtype=torch.int32, device=dev)
    I = torch.tensor([0], dtype=torch.int32, device=dev)
    G = torch.tensor([0], dtype=torch.int32, device=dev)
    out = torch.zeros((3, 1), dtype=torch.float64, device=dev)
    p = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(hh.HHError) as e:
        hh.hh_force_static(X, X, M, OFF, IDX, I, G, out, out, p)
    assert e.value.code == hh.HH_EINVAL and "131072" in str(e.value)
    # a list index outside [0, n_j) is caught on the device, nothing is written
    X2, M2 = X[:, :4].contiguous(), M[:4].contiguous()
    BAD = torch.tensor([0, 9], dtype=torch.int32, device=dev)
    out.fill_(7.0)
    with pytest.raises(hh.HHError) as e:
        hh.hh_force_static(X2, X2, M2, OFF, BAD, I, G, out, out, p)
    assert e.value.code == hh.HH_EINVAL
    assert torch.all(out == 7.0)
