"""Host logic of the performance-model module (the GPU analogue of the
paper's Table 1 and the Eq. 3 fit): the fit recovers known parameters and
the report carries the paper's rows."""
import numpy as np
import pytest

from paper_1602_02832_gb300 import perfmodel


def _rows(t_int, t_stage, n_is, n_ints, noise=0.0, seed=0):
    rng = np.random.default_rng(seed)
    rows = []
    for n_i, n_int in zip(n_is, n_ints):
        per = (t_int + t_stage / n_i) * (1.0 + noise * rng.standard_normal())
        rows.append({"form": "fp64", "n": 65536, "theta": 0.5, "n_crit": 64, "N_int": n_int, "n_i": n_i,
                     "T_force": per * n_int, "T_predict": 1e-8, "T_tree": 1e-9, "T_host": 1e-9,
                     "T_comm_round_trip": 1e-9})
    return rows


def test_fit_recovers_exact_parameters():
    rows = _rows(2.5e-11, 4.0e-10, [1.5, 3.0, 7.0, 12.0, 25.0], [2000, 2500, 11000, 5000, 22000])
    f = perfmodel.fit_force_model(rows)
    assert abs(f["t_int"] / 2.5e-11 - 1) < 1e-9
    assert abs(f["t_stage"] / 4.0e-10 - 1) < 1e-9
    assert abs(f["n_pipe"] - 16.0) < 1e-6
    assert f["r2"] > 0.999999 and f["points"] == 5


def test_fit_with_noise_is_close():
    rows = _rows(1e-10, 3e-9, np.linspace(1.2, 30, 40), np.full(40, 5000.0), noise=0.01, seed=3)
    f = perfmodel.fit_force_model(rows)
    assert abs(f["t_int"] / 1e-10 - 1) < 0.05
    assert abs(f["t_stage"] / 3e-9 - 1) < 0.05


def test_report_has_measured_fit_and_paper_rows():
    rows = _rows(2.5e-11, 4.0e-10, [2.0, 8.0], [3000, 9000])
    md = perfmodel.table_markdown(rows, {"fp64": perfmodel.fit_force_model(rows)})
    assert "| fp64 | 65536 | 0.5 | 64 |" in md
    for row in perfmodel.PAPER_TABLE1:
        assert f"| {row[0]} | {row[1]} | {row[2]} | {row[3]} |" in md
    # Table 1 values as printed in the paper (Section 3)
    assert perfmodel.PAPER_TABLE1[1][:4] == (65536, 0.5, 11081, 28.8)
    assert perfmodel.PAPER_TABLE1[5][:4] == (262144, 0.3, 28168, 29.4)


def test_static_tiles_follow_groups():
    # groups [0,5), [5,45), [45,46) with tile_i 16: runs of at most 16 inside each group
    gof = np.array([0] * 5 + [1] * 40 + [2])
    tiles = perfmodel._tiles(None, gof, 16)
    assert tiles == [(0, 5), (5, 21), (21, 37), (37, 45), (45, 46)]


def test_equivalent_performance_formula(monkeypatch):
    # S = 57 N n_step,h / T (Eq. 1): with a tree run of 1000 particle steps in
    # 1 ms and a direct run of 950 steps, S = 57 * 950 * N / 1e-3
    calls = []

    def fake_measure(n, theta, n_crit, precision, intervals, warm, seed):
        calls.append(theta)
        ps = 1000 if theta > 0 else 950
        per = 1e-6 if theta > 0 else 2e-5  # seconds per particle step, in T_force only
        return {"form": "fp64", "particle_steps": ps, "N_int": 2000.0 if theta > 0 else n - 1,
                "T_force": per, "T_predict": 0.0, "T_tree": 0.0, "T_host": 0.0}

    monkeypatch.setattr(perfmodel, "measure", fake_measure)
    e = perfmodel.equivalent_performance(4096, 0)
    assert calls == [0.5, 0.0]
    assert abs(e["S_tree_tflops"] - 57 * 950 * 4096 / 1e-3 / 1e12) < 1e-9
    assert abs(e["speedup_over_direct"] - (950 * 2e-5) / 1e-3) < 1e-12
    assert abs(e["steps_ratio_direct_over_tree"] - 0.95) < 1e-12


def test_list_run_stats_counts_runs_within_lists():
    from paper_1602_02832_gb300 import perfmodel
    # two lists: [0 1 2 | 5 6] [7 3 4 10 11] with n_particles = 10 (10, 11 are nodes);
    # 6 -> 7 crosses into the next list, so it starts a new run
    off = np.array([0, 5, 10])
    idx = np.array([0, 1, 2, 5, 6, 7, 3, 4, 10, 11])
    r = perfmodel.list_run_stats(off, idx, 10)
    assert r["entries"] == 10 and r["runs"] == 5  # [0 1 2] [5 6] [7] [3 4] [10 11]
    assert r["entries_per_run"] == 2.0
    assert r["particle_entries_per_run"] == 8 / 4 and r["node_entries_per_run"] == 2.0
    assert r["index_bytes_csr"] == 40 and r["index_bytes_ranges"] == 40
    assert r["index_share_of_staged_48B"] == pytest.approx(4 / 52)


def test_step_bins_sum_and_rates():
    # rows: active, interactions, list mode, step us, select + predict us, force us
    rows = np.array([[1, 100, 1, 10, 4, 6], [5, 300, 0, 12, 5, 7], [40, 4000, 0, 30, 10, 20],
                     [3000, 9e5, 0, 600, 20, 580], [5e5, 9e9, 0, 9e5, 50, 9e5 - 50]], dtype=float)
    b = perfmodel.step_bins(rows)
    assert [x["active"] for x in b][:3] == [[1, 8], [33, 128], [2049, 8192]]
    assert b[3]["active"][0] == 131073 and b[3]["steps"] == 1  # the largest steps have a bin too
    assert [x["steps"] for x in b] == [2, 1, 1, 1] and b[0]["list_steps"] == 1
    assert sum(x["time_share"] for x in b) == pytest.approx(1.0)
    assert sum(x["interaction_share"] for x in b) == pytest.approx(1.0)
    assert b[0]["force_us_sum"] == 13 and b[0]["select_predict_us_median"] == 4.5
    assert b[2]["force_rate"] == pytest.approx(9e5 / 580e-6)
