"""bench.py host logic on the CPU: argument handling, the workload record,
the algorithmic byte model and the reading of the committed ncu summaries."""
import sys

import pytest

import bench


def _args(monkeypatch, *argv):
    monkeypatch.setattr(sys, "argv", ["bench.py", *argv])
    return bench.parse()


def test_defaults_are_the_headline_workload(monkeypatch):
    a = _args(monkeypatch)
    assert (a.gpus, a.samples, a.grid, a.precision) == (1, 256, [64, 64, 16], "mixed")
    assert a.warmup >= 3 and a.steps >= 1
    assert a.predictor == 2 and a.smoother == "zline"
    cfg = bench.workload_config(a)
    assert cfg["workload"] == "elder3d-box-64x64x16-qmc256"
    assert cfg["nodes_per_sample"] == 65 * 65 * 17
    assert cfg["newton_start"] == "3u^n - 3u^(n-1) + u^(n-2)"


@pytest.mark.parametrize("argv,order", [(["--no-extrapolate"], 0), (["--predictor", "1"], 1),
                                        (["--predictor", "0"], 0)])
def test_predictor_flags(monkeypatch, argv, order):
    a = _args(monkeypatch, *argv)
    assert a.predictor == order
    assert bench.workload_config(a)["newton_start"].startswith(["u^n", "2u^n", "3u^n"][order])


def test_byte_model_matches_the_stored_formats():
    # mixed: bfloat16 multigrid matrices (108 entries x 2 B), FP32 vectors
    assert bench.E_model_bytes("mg_residual", 4, 64, 64, 16) == 108 * 2 + 6 * 4 + 1
    assert bench.E_model_bytes("spmv", 4, 64, 64, 16) == 108 * 4 + 6 * 4 + 1
    # z-line sweep from x = 0 with the assembly's line factors: zMi, zC, b, x
    # (FP32) and the lower line block (bfloat16)
    assert bench.E_model_bytes("smooth0", 4, 64, 64, 16) == 12 * 4 + 4 * 2 + 1
    # FP64: every stored entry 8 B
    assert bench.E_model_bytes("spmv", 8, 64, 64, 16) == 108 * 8 + 6 * 8 + 1


def test_traffic_lines_of_the_committed_profiles():
    assert bench.ncu_traffic("spmv", "mixed") == pytest.approx(428.0)
    assert bench.ncu_traffic("mg_residual", "mixed") == pytest.approx(229.8)
    assert bench.ncu_traffic("residual", "fp64") == pytest.approx(582.0)
    assert bench.ncu_traffic("no_such_class", "mixed") is None


def test_uneven_plan_covers_the_ensemble_once():
    """48 samples at 128x128x32 and 16 at 256x256x64: on one rank all of them,
    grouped by grid; on 4 ranks every sample exactly once, each rank's node
    count within 4/3 of the balanced share (the LPT bound)."""
    plan = bench.uneven_plan(1, 0)
    assert sorted(plan) == [(128, 128, 32), (256, 256, 64)]
    assert plan[(128, 128, 32)] == list(range(48)) and plan[(256, 256, 64)] == list(range(48, 64))
    nodes = {(128, 128, 32): 129 * 129 * 33, (256, 256, 64): 257 * 257 * 65}
    seen, loads = [], []
    for r in range(4):
        pl = bench.uneven_plan(4, r)
        loads.append(sum(nodes[g] * len(ids) for g, ids in pl.items()))
        seen += [i for ids in pl.values() for i in ids]
    assert sorted(seen) == list(range(64))
    total = 48 * nodes[(128, 128, 32)] + 16 * nodes[(256, 256, 64)]
    assert max(loads) <= 4 / 3 * total / 4


def _lobe_field(nx, ny, nz, centres, sigma=30.0, depth=93.75):
    """A node field [nz+1][ny+1][nx+1]: 1 on the top square, and below it
    Gaussian columns around the given (x, y) centres reaching `depth` m
    below the top."""
    import numpy as np
    x = np.linspace(0, 600, nx + 1)
    y = np.linspace(0, 600, ny + 1)
    z = np.linspace(0, 150, nz + 1)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    m = np.zeros_like(X)
    for xc, yc in centres:
        m = np.maximum(m, np.exp(-((X - xc) ** 2 + (Y - yc) ** 2) / (2 * sigma ** 2)) *
                       (Z >= 150 - depth))
    top = (X >= 150) & (X <= 450) & (Y >= 150) & (Y <= 450)
    m[-1] = np.where(top[-1], 1.0, 0.0)
    return m.ravel()


def test_plume_lobes_counts_five_fingers_at_the_corners_and_centre():
    pytest.importorskip("scipy")
    cen = [(150, 150), (450, 150), (150, 450), (450, 450), (300, 300)]
    r = bench.plume_lobes(_lobe_field(32, 32, 8, cen), 32, 32, 8)
    assert r["max_plane_count"] == 5
    assert sorted(l["nearest"] for l in r["plane"]["lobes"]) == sorted(
        ["corner(-,-)", "corner(+,-)", "corner(-,+)", "corner(+,+)", "centre"])
    for l in r["plane"]["lobes"]:
        assert min(abs(l["x_m"] - 150), abs(l["x_m"] - 300), abs(l["x_m"] - 450)) < 1e-6
    # planes deeper than the columns hold no lobe; the column-depth map sees
    # the five columns reaching 93.75 m, five cells (the top plane's square
    # does not count)
    assert r["plane_counts_top_down"][-1] == 0
    assert r["column_depth_max_m"] == pytest.approx(93.75)
    assert r["column_lobes_half_depth"] == 5


def test_plume_lobes_single_sheet_and_empty():
    pytest.importorskip("scipy")
    import numpy as np
    one = bench.plume_lobes(_lobe_field(32, 32, 8, [(300, 300)], sigma=120.0), 32, 32, 8)
    assert one["max_plane_count"] == 1 and one["plane"]["lobes"][0]["nearest"] == "centre"
    none = bench.plume_lobes(np.zeros(33 * 33 * 9), 32, 32, 8)
    assert none["max_plane_count"] == 0 and none["column_depth_max_m"] == 0.0
    assert none["column_lobes_half_depth"] == 0


def test_fingers_workload_defaults(monkeypatch):
    a = _args(monkeypatch, "--workload", "fingers")
    assert (a.fingers_samples, a.fingers_steps, a.fingers_grid, a.fingers_dt_yr) == \
        (200, 1500, [128, 128, 32], 0.005)


def test_compare_fingers_on_synthetic_fields(tmp_path):
    """Two field files of the same grid: one shifted by 0.01 at a quarter of
    the nodes; the comparison reports that difference, the lobe counts of
    both means and the variance level sets."""
    pytest.importorskip("scipy")
    import numpy as np
    nx, ny, nz = 32, 32, 8
    cen = [(150, 150), (450, 150), (150, 450), (450, 450), (300, 300)]
    m = _lobe_field(nx, ny, nz, cen).astype(np.float32)
    m2 = m.copy()
    m2[::4] += 0.01
    var = np.zeros_like(m)
    var[:100] = 0.06
    var2 = np.zeros_like(m)
    var2[:40] = 0.06
    a, b = tmp_path / "a.npz", tmp_path / "b.npz"
    np.savez(a, grid=np.array([nx, ny, nz]), mean_10=m, var=var)
    np.savez(b, grid=np.array([nx, ny, nz]), mean_10=m2, var=var2)
    out = bench.compare_fingers(str(a), str(b))
    assert out["snapshots"]["10"]["max_abs_dmean"] == pytest.approx(0.01, rel=1e-3)
    assert out["plane_counts_top_down"]["a"] == out["plane_counts_top_down"]["b"]
    assert max(out["plane_counts_top_down"]["a"]) == 5
    assert out["var_level_set"] == {"level": 0.05, "a": 100, "b": 40, "both": 40}


def test_reference_arm_line_on_a_tiny_grid():
    """bench.py --impl reference on a 4x4x2 grid with 2 worker processes: one
    JSON line with the reference keys (impl, cpu_baseline with its cores and
    sample, an e2e object with zero copy bytes) and a positive rate."""
    import json
    import os
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--grid", "4", "4", "2",
                          "--steps", "3", "--warmup", "1", "--cpu-workers", "2"],
                         cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["cores"] == 2 and line["cpu_baseline"]["kind"] == "oracle"
    assert "4 sample-steps" in line["cpu_baseline"]["sample"]   # 3 steps -> 2 whole rounds of 2
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["higher_is_better"] is True and line["unit"] == bench.UNIT
