"""hh_force_static, the allocation-free force call, on the GPU.

Some callers cannot allocate device memory: their memory all comes from
another allocator or pool, or their loop must not call cudaMalloc / cudaFree,
which synchronise the whole device.  hh_force_static serves them from one fixed
scratch array inside libhh.  This file checks, through the C ABI:
- two calls in a row give the same forces as the regular hh_force path, and
  both meet the per-particle bars against the FP64 oracle (tests/_parity.py:
  FP64 1e-11; mixed acc and pot 1e-6, jerk 1e-5 or 1e-6 of J_scale);
- device memory in use does not change across calls after the first;
- sizes beyond the fixed limits, too many work items, list ids outside
  [0, n_groups) and list indices outside [0, n_j) are refused with the
  documented codes, and the outputs keep their previous contents.
It sits in its own file, collected last, and passes alone or after the other
tests.
"""
import numpy as np
import pytest

import _parity
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
    ins = [(torch.tensor(ia, device=dev), torch.tensor(T.group_of[ia], device=dev)) for ia in sets]
    outs = [(torch.zeros((3, len(ia)), dtype=torch.float64, device=dev),
             torch.zeros((3, len(ia)), dtype=torch.float64, device=dev),
             torch.zeros(len(ia), dtype=torch.float64, device=dev)) for ia in sets]
    # the first call on the device sets up the scratch (module load, symbol
    # address); from then on no call may change the device memory in use
    hh.hh_force_static(X, V, M, OFF, IDX, *ins[1], *outs[1], eps2=eps2, precision=P)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(0)[0]
    got = []
    for (I, G), (acc, jerk, pot) in zip(ins, outs):  # two calls in a row, different active sets
        hh.hh_force_static(X, V, M, OFF, IDX, I, G, acc, jerk, pot, eps2=eps2, precision=P)
        got.append((acc.cpu().numpy(), jerk.cpu().numpy(), pot.cpu().numpy()))
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info(0)[0]
    assert free1 == free0, (free0, free1)
    with hh.Context(cfg, n, nj, len(T.list_idx), T.n_groups) as ctx:
        ctx.hh_set_j(0, xj.T, vj.T, aj.T, jj.T, mj, np.zeros(nj))
        ctx.hh_set_lists(n, nj, T.list_off, T.list_idx, T.group_of)
        ctx.hh_predict(0.0)
        refs = [ctx.hh_force(ia) for ia in sets]
    for ia, g, ref in zip(sets, got, refs):
        # same kernel, same list parts: equal to hh_force up to the tile
        # boundaries of the active set (FP64 reordering, FP32 rounding)
        lim = 1e-11 if P == hh.HH_FP64 else 1e-6
        assert _rel(g[0], ref[0]).max() < lim and _rel(g[1], ref[1]).max() < 10 * lim
        assert (np.abs(g[2] - ref[2]) / np.abs(ref[2])).max() < lim
        ra, rj, rp = orc.list_force(xj, vj, mj, ia, T.group_of[ia], T.list_off, T.list_idx, eps2)
        _parity.check(P == hh.HH_FP64, *g, ra, rj, rp,
                      lambda k, ia=ia: _parity.jscale(xj, vj, mj, T.group_of[ia[k]], T.list_off, T.list_idx,
                                                      ia[k], eps2),
                      f"{prec} hh_force_static, {len(ia)} active")


def _tiny(torch, dev, n_act, gid_of):
    X = torch.zeros((3, 4), dtype=torch.float64, device=dev)
    X[0] = torch.arange(4, dtype=torch.float64, device=dev)
    M = torch.ones(4, dtype=torch.float64, device=dev)
    OFF = torch.tensor([0, 2, 4], dtype=torch.int64, device=dev)
    IDX = torch.tensor([0, 1, 2, 3], dtype=torch.int32, device=dev)
    I = torch.tensor(np.arange(n_act) % 4, dtype=torch.int32, device=dev)
    G = torch.tensor(gid_of(np.arange(n_act)), dtype=torch.int32, device=dev)
    acc = torch.full((3, n_act), 7.0, dtype=torch.float64, device=dev)
    jerk = torch.full((3, n_act), 7.0, dtype=torch.float64, device=dev)
    pot = torch.full((n_act,), 7.0, dtype=torch.float64, device=dev)
    return X, M, OFF, IDX, I, G, acc, jerk, pot


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
    out2 = torch.zeros((3, 1), dtype=torch.float64, device=dev)
    p = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(hh.HHError) as e:
        hh.hh_force_static(X, X, M, OFF, IDX, I, G, out, out2, p)
    assert e.value.code == hh.HH_EINVAL and "131072" in str(e.value)
    # a list index outside [0, n_j) is caught on the device, nothing is written
    X2, M2 = X[:, :4].contiguous(), M[:4].contiguous()
    BAD = torch.tensor([0, 9], dtype=torch.int32, device=dev)
    out.fill_(7.0)
    with pytest.raises(hh.HHError) as e:
        hh.hh_force_static(X2, X2, M2, OFF, BAD, I, G, out, out2, p)
    assert e.value.code == hh.HH_EINVAL
    assert torch.all(out == 7.0)


def test_force_static_device_detected_errors_leave_outputs(env):
    hh, torch, _ = env
    dev = torch.device("cuda", 0)
    # 8193 actives alternating between two lists: every active is its own
    # tile, one work item each, one above the 8192-item capacity
    X, M, OFF, IDX, I, G, acc, jerk, pot = _tiny(torch, dev, 8193, lambda k: k % 2)
    with pytest.raises(hh.HHError) as e:
        hh.hh_force_static(X, X, M, OFF, IDX, I, G, acc, jerk, pot)
    assert e.value.code == hh.HH_ENOMEM
    assert torch.all(acc == 7.0) and torch.all(jerk == 7.0) and torch.all(pot == 7.0)
    # a list id equal to n_groups (outside [0, n_groups))
    X, M, OFF, IDX, I, G, acc, jerk, pot = _tiny(torch, dev, 3, lambda k: np.where(k == 1, 2, 0))
    with pytest.raises(hh.HHError) as e:
        hh.hh_force_static(X, X, M, OFF, IDX, I, G, acc, jerk, pot)
    assert e.value.code == hh.HH_EINVAL
    assert torch.all(acc == 7.0) and torch.all(jerk == 7.0) and torch.all(pot == 7.0)
    # and the scratch is usable again: 8192 items exactly is accepted
    X, M, OFF, IDX, I, G, acc, jerk, pot = _tiny(torch, dev, 8192, lambda k: k % 2)
    hh.hh_force_static(X, X, M, OFF, IDX, I, G, acc, jerk, pot)
    a = acc.cpu().numpy()
    assert np.all(np.isfinite(a)) and not np.any(a == 7.0)
    # particle at x = 0 (index 0, list 0 = entries {0, 1}): pulled towards x = 1
    assert a[0, 0] > 0
