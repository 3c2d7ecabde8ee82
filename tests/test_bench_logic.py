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
