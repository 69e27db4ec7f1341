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
    assert (a.workload, a.restart, a.reorth, a.coarse_max, a.gpus) == ("layered128", 20, 0, 512, 1)
    assert a.warmup >= 3
    a = _args(monkeypatch, "--workload", "lognormal64")
    assert a.restart == 12
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


def test_operator_flops_and_step_bytes():
    # one cell: 8 nodes all coupled (64 3x3 blocks), 24 + 24 coupling
    # entries, 4 p-block and 12 cell-face entries, 6 faces x 11 ELL slots
    assert bench.operator_flops(1) == 2 * (576 + 48 + 4 + 12 + 66)
    hu, hpi = [274625, 10648, 512], [798720, 262144, 10648, 512]
    b32 = bench.step_bytes(64, hu, hpi, 1, 12, 32)
    b64 = bench.step_bytes(64, hu, hpi, 0, 12, 32)
    assert b64 > b32 > 0                       # FP64 V-cycles move more bytes
    # one more iteration adds at least one operator apply and one preconditioner
    op = 27 * 9 * 8 * 65 ** 3
    assert bench.step_bytes(64, hu, hpi, 1, 12, 33) - b32 > op
    # a longer restart does more Gram-Schmidt work for the same iterations
    assert bench.step_bytes(64, hu, hpi, 1, 32, 32) > b32


def test_cpu_legs_scaling_rule():
    # two cores, each 1e5 unknowns x 10 iterations in 2 s: 1e6 (unknown x
    # iteration) / s in total; the full workload at 54 iterations
    step = [(24, 100000, 10, 2.0), (24, 100000, 10, 2.0)]
    n_full = sum(bench.make_problem_sizes("layered128"))
    assert bench.full_estimate_ms("layered128", step, 54) == pytest.approx(n_full * 54 / 1e6 * 1e3)


def test_oracle_leg_runs_on_spawned_processes():
    """The CPU leg's process fan-out on a tiny sample: two spawned oracle
    processes step together; every step reports both, with the oracle's own
    iteration counts."""
    steps = bench.oracle_leg("lognormal32", [3, 4], 2)
    assert len(steps) == 2
    for st, wall in steps:
        assert [s[0] for s in st] == [3, 4] and wall > 0
        assert all(it > 0 and sec > 0 for _, _, it, sec in st)
        assert st[1][1] == sum(bench.make_problem_sizes_n("lognormal32", 4))
