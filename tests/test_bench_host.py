"""bench.py's host logic (no GPU): workload defaults, option pass-through,
sizes and the arithmetic behind the reported roofline figures."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _args(monkeypatch, *argv):
    monkeypatch.setattr(sys, "argv", ["bench.py", *argv])
    return bench.parse()


def test_workload_defaults(monkeypatch):
    a = _args(monkeypatch)
    assert (a.workload, a.restart, a.reorth, a.coarse_max, a.gpus) == ("lognormal64", 12, 0, 512, 1)
    assert a.warmup >= 3
    a = _args(monkeypatch, "--workload", "layered128")
    assert a.restart == 20
    a = _args(monkeypatch, "--workload", "layered128", "--restart", "7", "--reorth", "1", "--coarse-max", "125")
    assert (a.restart, a.reorth, a.coarse_max) == (7, 1, 125)


def test_sizes_and_roofline_arithmetic():
    assert bench.make_problem_sizes("lognormal64") == (3 * 65 ** 3, 64 ** 3, 3 * 64 * 64 * 65)
    assert sum(bench.make_problem_sizes("layered128")) == 14877827
    # 152 SMs x 2 FP64 FMA per clock x 2 flop at 2070 MHz
    assert bench.fp64_peak_tflops(2070.0) == pytest.approx(1.25856)
    # one FP64 sweep on a 1-cell mesh: 8 nodes, each coupled to all 8 (3x3 blocks)
    assert bench.cheb_u0_flops(1) == 2 * 9 * 64 + 2 * 9 * 8 + 4 * 3 * 8
    # whole-job time per step of N independent replicas
    assert bench.aggregate_time(40.0, 4) == 10.0
