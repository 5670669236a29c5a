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
    assert bench.E_model_bytes("smooth0", 4, 64, 64, 16) == 8 * 4 + 1 + 8 * 2
    # FP64: every stored entry 8 B
    assert bench.E_model_bytes("spmv", 8, 64, 64, 16) == 108 * 8 + 6 * 8 + 1


def test_traffic_lines_of_the_committed_profiles():
    assert bench.ncu_traffic("spmv", "mixed") == pytest.approx(436.3)
    assert bench.ncu_traffic("mg_residual", "mixed") == pytest.approx(229.8)
    assert bench.ncu_traffic("residual", "fp64") == pytest.approx(302.0)
    assert bench.ncu_traffic("no_such_class", "mixed") is None
