"""Host-side helpers of bench.py: latency percentiles (block steps in
microseconds, requests in seconds), the active-particles-per-tile summary
(the paper's n_i) and the per-interval time split."""
import numpy as np
import pytest

import bench


def test_latency_percentiles_and_notes():
    lat = bench._lat([4.0, 1.0, 3.0, 2.0])
    assert lat["p50"] == pytest.approx(2.5)
    assert lat["p99"] == pytest.approx(np.quantile([1, 2, 3, 4], 0.99))
    assert lat["mean"] == pytest.approx(2.5) and lat["n"] == 4
    assert "block step" in lat["note"]
    req = bench._lat([0.5, 1.5], "wall seconds from a request's arrival to its completion")
    assert req["p50"] == pytest.approx(1.0) and "request" in req["note"]
    assert bench._lat([]) is None


def test_active_per_tile_summary():
    # counts[k] tiles had k + 1 active particles
    s = bench._n_i({"n_i_hist": [2, 1, 0, 1] + [0] * 28})
    assert s["tiles"] == 4
    assert s["mean"] == pytest.approx((1 * 2 + 2 * 1 + 4 * 1) / 4)
    assert s["counts"] == [2, 1, 0, 1]  # trailing empty bins dropped
    assert bench._n_i({"n_i_hist": [0] * 32}) is None
    assert bench._n_i({}) is None


def test_time_split_per_interval():
    r = {"ms": 10.0, "force_ms": 6.0, "phase_ms": [1.0, 6.0, 0.0]}
    s = bench._split(r, 2)
    assert s == pytest.approx({"predict_select": 0.5, "force": 3.0, "correct": 0.0, "rebuild_and_launch": 1.5})
    # the graph loop times only the force kernel
    s = bench._split({"ms": 10.0, "force_ms": 6.0, "phase_ms": [0.0, 0.0, 0.0]}, 2)
    assert s == pytest.approx({"force_kernel": 3.0, "other": 2.0})


def test_reference_arm_prints_one_contract_line():
    # the oracle arm on the host cores: one JSON line with the contract's keys;
    # a rank other than 0 exits without work
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--n", "1024", "--steps", "2",
           "--warmup", "1"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, check=True, cwd=root)
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=root)
    assert r.returncode == 0 and not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_traffic_is_reported_only_for_the_captured_kernel_sources(monkeypatch):
    shape = dict(bench.TRAFFIC_FP64["shape"])
    assert set(shape) == set(bench.SHAPE_KEYS)
    monkeypatch.setitem(bench.TRAFFIC_FP64, "bytes", 123.0)
    monkeypatch.setitem(bench.TRAFFIC_FP64, "sources_sha16", bench._sources_sha16())
    assert bench._traffic(shape) == 123.0
    assert bench._traffic(dict(shape, tile_j=512)) is None  # another tile shape
    monkeypatch.setitem(bench.TRAFFIC_FP64, "sources_sha16", "0" * 16)
    assert bench._traffic(shape) is None
    monkeypatch.setitem(bench.TRAFFIC_FP64, "bytes", None)
    assert bench._traffic(shape) is None


def test_cpu_leg_resumes_the_given_state_and_checks_sampled_forces(orc):
    # the CPU baseline starts the oracle from the state it is handed (the GPU
    # arm's, at the start of its timed window) and, given config-3 data,
    # compares the handed forces with the oracle's list force
    import synth

    n = 600
    x, v, m = synth.plummer(n, 4)
    a = bench._args(["--n", str(n), "--n-crit", "32"])
    p = bench._oracle_params(a)
    r = orc.run(x, v, m, p.dt_tree, p)
    state = {"x": r["x"], "v": r["v"], "a": r["a"], "jk": r["jk"], "dt": r["dt"], "m": m, "t": p.dt_tree}
    T = orc.tree_build(r["x"], r["v"], r["a"], r["jk"], m, leaf=8, n_crit=32, theta=0.5)
    xj, vj, aj, jj, mj = T.j_array(r["x"], r["v"], r["a"], r["jk"], m)
    s = np.arange(0, n, 7, dtype=np.int32)
    ra, rj, rp = orc.list_force(xj, vj, mj, s, T.group_of[s], T.list_off, T.list_idx, 1e-8)
    gpu = (ra.T * (1 + 1e-9), rj.T, rp)
    cfg3 = {"xj": xj, "vj": vj, "mj": mj, "off": T.list_off, "idx": T.list_idx, "gof": T.group_of, "sample": s,
            "gpu": gpu}
    out = bench._cpu_baseline(a, state, cfg3)
    assert out["value"] > 0 and out["kind"] == "oracle" and out["cores"] >= 1
    assert f"t = {p.dt_tree:g}" in out["sample"]
    ck = out["config3_check"]
    assert ck["particles"] == len(s)
    assert ck["acc_max_rel"] == pytest.approx(1e-9, rel=1e-3)
    assert ck["jerk_max_rel"] == 0.0 and ck["pot_max_rel"] == 0.0


def test_latency_by_live_count_bins():
    out = bench._lat_by_live([10.0, 20.0, 30.0, 40.0, 50.0], [1, 1, 2, 3, 5])
    assert [b["live"] for b in out] == [[1, 1], [2, 3], [4, 7]]
    assert [b["steps"] for b in out] == [2, 2, 1]
    assert out[0]["p50_us"] == pytest.approx(15.0) and out[2]["p99_us"] == pytest.approx(50.0)
    assert bench._lat_by_live([], []) is None


def test_queue_by_quarter_and_latency_by_size():
    q = [(0.5, 0, 1), (1.0, 2, 3), (3.0, 4, 5), (3.5, 6, 7), (7.9, 1, 1)]
    out = bench._queue_by_quarter(q, 8.0)
    assert [b["launches"] for b in out] == [2, 2, 0, 1]
    assert out[0]["waiting_mean"] == 1.0 and out[1]["resident_mean"] == 6.0
    assert out[2]["waiting_mean"] is None and out[3]["waiting_mean"] == 1.0

    class R:
        def __init__(self, rid, arrival_s, done_s):
            self.rid, self.arrival_s, self.done_s = rid, arrival_s, done_s

    n_of = {0: 1024, 1: 4095, 2: 4096, 3: 1 << 18}
    res = [R(0, 0.0, 1.0), R(1, 0.0, 3.0), R(2, 1.0, 2.0), R(3, 0.0, 9.0)]
    by = bench._lat_by_n(res, n_of)
    assert [b["n"] for b in by] == [[1024, 4095], [4096, 16383], [65536, 1 << 18]]
    assert by[0]["completed"] == 2 and by[0]["max_s"] == 3.0
    assert by[2]["p50_s"] == 9.0
    assert bench._lat_by_n([], n_of) is None
