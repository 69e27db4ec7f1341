#!/usr/bin/env python3
"""Time-to-solve per backward-Euler step of the stabilized hybridized
poromechanics system (FGMRES + block-triangular multigrid preconditioner,
FP64) on one GB300, to a 1e-8 relative residual of the equilibrated system.

Default workload: the largest single-GPU configuration, 128^3 unit cube
with interior node jitter U(+-0.2h), 8 horizontal layers (kappa log-U
[1e-18, 1e-12] m^2, E log-U[1e8, 1e10] Pa, nu U[0.2, 0.35]), S_eps = 0,
dt = 0.1 s, consolidation-column boundaries; 14,877,827 unknowns.  The 64^3
log-normal workload (1,884,739 unknowns) is measured in the same run and
reported inside config.  A "step" is one time step: right-hand side from
the previous state + FGMRES solve.
The operator and the preconditioner are built once (constant dt), timed
separately as setup_ms.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU runs (torchrun) solve independent replicas, one per rank.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-solve per step to 1e-8 rel. residual"
TOL = 1e-8
FALLBACK_HBM_GBS = 6800.0

# gpu_iters: FGMRES iterations per step the GPU solve takes on the workload
# (measured; the CPU legs scale their samples to it, the oracle being the
# same algorithm)
WORKLOADS = {
    "lognormal64": dict(n=64, restart=12, gpu_iters=35,
                        desc="64^3 hex, log-normal kappa (sigma 2, corr. 8 cells, seed 2), S_eps=0, dt=1e-3 s"),
    "lognormal32": dict(n=32, gpu_iters=28,
                        desc="32^3 hex, log-normal kappa (sigma 2, corr. 8 cells, seed 2), S_eps=0, dt=1e-3 s"),
    "lognormal96": dict(n=96, gpu_iters=36,
                        desc="96^3 hex, log-normal kappa (sigma 2, corr. 8 cells, seed 2), S_eps=0, dt=1e-3 s"),
    "layered128": dict(n=128, gen="layered", restart=20, gpu_iters=56,
                       desc="128^3 hex, interior node jitter U(+-0.2h), 8 z-layers: kappa log-U[1e-18,1e-12] m^2, "
                            "E log-U[1e8,1e10] Pa, nu U[0.2,0.35]; S_eps=0, dt=0.1 s (seed 3)"),
    "adjoint48": dict(n=48, desc="48^3 hex, log-normal ln kappa (sigma 1, seed 5), 10 backward-Euler steps dt=0.1 s, "
                                 "misfit of top u_z and cell p against a second seeded field; J and dJ/d ln kappa "
                                 "(110,592 cells) by the checkpointed discrete adjoint, solves to 1e-10"),
    "cantilever_can3": dict(n=0, desc="Test 2 cantilever (unit cube clamped at x=0, unit load on top, no-flow, E=1e5 Pa, "
                                      "nu=0.4, kappa=1e-7 m^2, mu=1e-3 Pa s) at 1/h = 64, 128 and 256, dt = 0.1 and "
                                      "1e-5 s: M_II^(m) (mixed form) beside M_II^(h) and M_III^(h), FP64, FGMRES(30), "
                                      "tol 1e-6"),
    "batch48": dict(n=0, desc="48 cubes n ~ U{16..64} (seed 4), own log-normal kappa (sigma 1.5), loads x0.5/1/2/4, "
                              "FP32 V-cycles in FP64 FGMRES(12), all 192 systems in one CUDA graph launch"),
}


def make_problem(name, n=None):
    """The workload's problem, or the same generator at n^3 (oracle samples)."""
    import mhfp_inputs as mi
    n = WORKLOADS[name]["n"] if n is None else n
    if WORKLOADS[name].get("gen") == "layered":
        return mi.layered_jitter_cube(n)
    return mi.lognormal_cube(n)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="layered128")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-64", action="store_true", help="skip the 64^3 workload measured beside the 128^3 one")
    ap.add_argument("--can3-grids", default="64,128,256",
                    help="1/h values of the cantilever_can3 workload (comma separated)")
    ap.add_argument("--restart", type=int, default=None,
                    help="FGMRES restart length (default: the fastest measured for the workload, 12 at 64^3, "
                         "20 at 128^3)")
    ap.add_argument("--coarse-max", type=int, default=512,
                    help="coarsen while a multigrid level has more lattice points (512: the 64^3 workload's "
                         "hierarchies end at 8^3 points, inverted densely on the GPU)")
    ap.add_argument("--reorth", type=int, choices=[0, 1], default=0,
                    help="Gram-Schmidt: 0 one classical pass (PETSc's GMRES default; same iterations and "
                         "residuals on the workloads), 1 DGKS reorthogonalisation when needed")
    ap.add_argument("--cheb-degree", type=int, default=0, choices=[0, 1, 2, 3],
                    help="Chebyshev smoother degree; 0 (default): chosen by the set-up autotuner, which solves the "
                         "step's load with degrees 1-3 and keeps the fastest")
    ap.add_argument("--precision", choices=["both", "mixed", "fp64"], default="both",
                    help="both: mixed headline with FP64-plain beside it (default)")
    args = ap.parse_args()
    if args.restart is None:
        args.restart = WORKLOADS[args.workload].get("restart", 12)
    return args


SINGLE_THREAD_ENV = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1",
                     "NUMEXPR_NUM_THREADS": "1"}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_worker(workload, sample_n, seed_shift, nsteps, barrier, out):
    """One host core's share of the oracle leg: the workload's generator at
    sample_n^3 (assembly and preconditioner set-up untimed), then `nsteps`
    backward-Euler steps, each started at the shared barrier and timed."""
    for k, v in SINGLE_THREAD_ENV.items():
        os.environ[k] = v
    import oracle
    from oracle import fgmres, precond, system
    prob = make_problem(workload, sample_n)
    B = oracle.assemble(prob)
    pc = precond.build(B, "amg", coarse_max=512)
    A = system.system_matrix(B)
    sc = precond.equilibration(B, pc.Bt, pc.C)
    nU, nP, _ = B.sizes
    n_s = sum(B.sizes)
    m = WORKLOADS[workload].get("restart", 12)
    xprev = None
    for k in range(nsteps):
        barrier.wait()
        t0 = time.perf_counter()
        b = system.rhs(B, None if xprev is None else xprev[:nU], None if xprev is None else xprev[nU:nU + nP])
        x, info = fgmres.fgmres(lambda v: A @ v, pc.apply, b, tol=TOL, restart=m, scale=sc)
        out.put((seed_shift, k, sample_n, n_s, info["iters"], time.perf_counter() - t0))
        xprev = x


def oracle_leg(workload, samples, nsteps, on_step=None):
    """Run the oracle as it stands on the host cores: one spawned process
    per entry of `samples` (a sample size each), all stepping together.
    Returns per step a list of (sample_n, unknowns, iterations, seconds) and
    the step's wall time."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(len(samples) + 1)
    out = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(workload, n, i, nsteps, barrier, out), daemon=True)
             for i, n in enumerate(samples)]
    for p in procs:
        p.start()
    steps = []
    try:
        for k in range(nsteps):
            barrier.wait(timeout=900)
            t0 = time.perf_counter()
            got = [out.get(timeout=900) for _ in samples]
            wall = time.perf_counter() - t0
            steps.append(([g[2:] for g in sorted(got)], wall))
            if on_step:
                on_step(k, steps[-1])
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    return steps


def full_estimate_ms(workload, step, iters_full):
    """The oracle's time for one step of the full workload from a step of
    concurrent samples: every core's rate (unknowns x FGMRES iterations per
    second) measured while all cores run, summed, and the full workload's
    unknowns x iterations divided by it (the same rule for both CPU legs;
    the full workload's iteration count is the GPU's, the same algorithm)."""
    rate = sum(n_s * it / sec for _, n_s, it, sec in step)
    n_full = sum(make_problem_sizes(workload))
    return n_full * iters_full / rate * 1e3


def cpu_baseline_leg(workload, iters_full):
    """cpu_baseline of our arm: one step of the oracle on every host core at
    the 32^3 sample of the workload's generator, plus one core at 48^3 to
    check that the cost per unknown and iteration holds as the sample grows."""
    cores = host_cores()
    ncore = max(1, min(cores, 16))
    samples = [48] + [32] * (ncore - 1) if ncore > 1 else [32]
    t0 = time.perf_counter()
    (step, wall), = oracle_leg(workload, samples, 1)
    total = time.perf_counter() - t0
    per = {}
    for n_s_mesh, n_s, it, sec in step:
        per.setdefault(n_s_mesh, []).append((n_s, it, sec))
    cost = {f"{k}^3": {"unknowns": v[0][0], "iterations": v[0][1],
                       "us_per_unknown_iteration": 1e6 * statistics.mean(sec / (n_s * it) for n_s, it, sec in v)}
            for k, v in per.items()}
    value = full_estimate_ms(workload, step, iters_full)
    return {"value": value, "unit": "ms", "cores": len(samples), "kind": "oracle",
            "extrapolated": True,
            "sample": (f"one backward-Euler step of the workload's generator on each of {len(samples)} host "
                       f"processes (one per core, one BLAS thread each; {samples.count(32)} at 32^3, "
                       f"{samples.count(48)} at 48^3), assembly and set-up untimed, {wall:.1f} s of wall time; "
                       f"the summed per-core rate (unknowns x FGMRES iterations / s) scaled to the full "
                       f"workload's unknowns x the GPU's {iters_full:.0f} iterations"),
            "oracle_iterations_in_sample": {k: v["iterations"] for k, v in cost.items()},
            "cost_per_unknown_iteration": cost, "leg_seconds": total}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------------ clocks
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def clocks_start(dev_index):
    f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    try:
        p = subprocess.Popen(["nvidia-smi", f"--id={dev_index}", f"--query-gpu={CLOCK_Q}",
                              "--format=csv,noheader,nounits", "-lms", "200"], stdout=f,
                             stderr=subprocess.DEVNULL)
    except (OSError, FileNotFoundError):
        return None, f.name
    return p, f.name


def clocks_stop(proc, path):
    if proc is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [s.strip() for s in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax.append(float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    os.unlink(path)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle
def run_reference(args):
    """--impl reference: the oracle as it stands on the host cores (one
    process per core), each step one backward-Euler step of every process's
    24^3 sample of the workload's generator; the step's time is scaled to the
    full workload by the rule of full_estimate_ms, with the full workload's
    iteration count the GPU's measured one for this workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_full = sum(make_problem_sizes(args.workload))
    iters_full = WORKLOADS[args.workload]["gpu_iters"]
    ncore = max(1, min(host_cores(), 16))
    samples = [24] * ncore
    steps = oracle_leg(args.workload, samples, args.warmup + args.steps)
    timed = steps[args.warmup:]
    per_step = [full_estimate_ms(args.workload, st, iters_full) for st, _ in timed]
    walls = [w for _, w in timed]
    its = sorted({it for st, _ in timed for _, _, it, _ in st})
    ms = sum(per_step) / len(per_step)
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"], "unknowns": n_full, "tol": TOL,
                       "parallelism": "replicas"},
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": ncore, "kind": "oracle", "extrapolated": True,
                             "sample": (f"each step = one backward-Euler step on each of {ncore} host processes "
                                        f"(one per core, one BLAS thread each) of the workload's generator at "
                                        f"24^3 ({sum(make_problem_sizes_n(args.workload, 24))} unknowns, oracle "
                                        f"FGMRES iterations {its}), {statistics.mean(walls):.2f} s of wall time "
                                        f"per step; the summed per-core rate scaled to the full workload's "
                                        f"{n_full} unknowns x {iters_full} iterations (the GPU's count)"),
                             "wall_s_per_step": statistics.mean(walls)},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def make_problem_sizes(name):
    return make_problem_sizes_n(name, WORKLOADS[name]["n"])


def make_problem_sizes_n(name, n):
    return (3 * (n + 1) ** 3, n ** 3, 3 * n * n * (n + 1))


def traffic_for(kernel, workload, bytes_per_launch):
    """DRAM read+write bytes per launch of `kernel` from the committed ncu
    summary (profiles/traffic.json), scaled to this workload's launch by the
    ratio of algorithmic bytes when the capture ran on a smaller case; None
    if there is no capture or the kernel's source region changed since."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel)
    if not d:
        return None
    src = open(os.path.join(ROOT, "paper_2002_09603_gb300", "csrc", d["source"])).read()
    tag = d["region"]
    try:
        a, b = src.index(f"// <{tag}>"), src.index(f"// </{tag}>")
    except ValueError:
        return None
    sha = hashlib.sha256(src[a:b].encode()).hexdigest()[:16]
    if sha != d["region_sha"]:
        return None
    if d.get("workload", "lognormal64") == workload or not d.get("algorithmic_bytes"):
        return d["bytes_per_launch"] if d.get("workload", "lognormal64") == workload else None
    return d["bytes_per_launch"] * bytes_per_launch / d["algorithmic_bytes"]


# FP64 peak of the part: ~2 FP64 FMA per clock per SM (from the pipe
# utilisation ncu reports for k_cheb_u0), 152 SMs, 2 flop per FMA, at the
# maximum SM clock -> 1.26 TFLOP/s (nominal GB300 FP64: 1.25 TFLOP/s).
FP64_FMA_PER_CLK_SM = 2
N_SM = 152


def fp64_peak_tflops(sm_max_mhz):
    return N_SM * FP64_FMA_PER_CLK_SM * 2 * sm_max_mhz * 1e6 / 1e12


def cheb_u0_flops(n):
    """Algorithmic FP64 flops of one k_cheb_u0 launch on an n^3 mesh:
    2 per FMA of r = b - A x over the valid (node, neighbour) 3x3 blocks,
    of D^-1 r, and 4 per dof for the two Chebyshev updates."""
    L = n + 1
    blocks = (3 * L - 2) ** 3
    nodes = L ** 3
    return 2 * 9 * blocks + 2 * 9 * nodes + 4 * 3 * nodes


def operator_flops(n):
    """Algorithmic FP64 flops of one operator apply A_H x on an n^3 mesh:
    2 per stored coefficient the three row kernels multiply -- A_uu's valid
    (node, neighbour) 3x3 blocks, A_up and A_pu (24 per cell each), the
    p-block (diagonal and three macro partners per cell), A_ppi and A_pip
    (6 per cell each) and the 11 ELL slots of A_pipi per face."""
    L = n + 1
    nT, nF = n ** 3, 3 * n * n * L
    nnz = 9 * (3 * L - 2) ** 3 + 48 * nT + 4 * nT + 12 * nT + 11 * nF
    return 2 * nnz


# ------------------------------------------------------ step-level bytes
# Algorithmic HBM bytes of one time step (each stored value, inverse
# diagonal block and vector touched once per kernel; coarse levels counted
# the same way although they sit in L2).  Per lattice level of N points
# with b unknowns per point, K stencil offsets and s bytes per value:
# values V = K b^2 s (the finest FP32 displacement level stores the
# symmetric half, 14 of 27 blocks), inverse diagonal D = b^2 s, a vector
# v = b s per point.
STENCIL = {"box1": 27, "diamond2": 25, "box2": 125, "faces": 11}


def _vcycle_bytes(levels, s, fine_sym):
    """One V(1,1) cycle with Chebyshev(2) smoothing: per non-last level a
    zero-start step (D + 3v), three stencil steps (V + D + 5v each), a
    residual (V + 3v), the restriction and prolongation (prolongator values
    or face weights plus 3v); the last level is the FP64 dense inverse
    (n^2 x 8 B) and two vectors."""
    total = 0.0
    for i, (kind, N, b) in enumerate(levels):
        v, D = b * s * N, b * b * s * N
        if i == len(levels) - 1:
            n = N * b
            total += n * n * 8 + 2 * v
            break
        K = 14 if (fine_sym and i == 0) else STENCIL[kind]
        V = K * b * b * s * N
        slots = 8 if kind == "box1" else 27
        Pb = (s * N) if kind == "faces" else slots * b * b * s * N
        total += (D + 3 * v) + 3 * (V + D + 5 * v) + (V + 3 * v) + 2 * (Pb + 3 * v)
    return total


def step_bytes(n_mesh, hu_points, hpi_points, precision, m, iters_per_step):
    """Algorithmic bytes of one time step (right-hand side + FGMRES solve).

    Per Arnoldi step j: the preconditioner (precision conversions, the
    interface-pressure V-cycle, the two Schur steps, the displacement
    V-cycle), the operator (float-float in the mixed form), one classical
    Gram-Schmidt pass over the
    j + 1 basis vectors (dots, update, normalisation) and the Givens step.
    Per restart cycle: the residual (operator + norm) and x += Z y."""
    L = n_mesh + 1
    nN, nT = L ** 3, n_mesh ** 3
    nF = 3 * n_mesh * n_mesh * L
    n = 3 * nN + nT + nF
    s = 4 if precision == 1 else 8
    hu = [("box1", N, 3) for N in hu_points]
    hpi = [("faces", hpi_points[0], 1)] + [("diamond2" if i == 1 else "box2", N, 1)
                                           for i, N in enumerate(hpi_points) if i > 0]
    conv = (20 + 12) * n if precision == 1 else 24 * n
    schur = (6 * s + 3 * s) * nT + nF * s + 24 * s * nT + s * nT + 6 * s * nN
    prec = conv + _vcycle_bytes(hpi, s, False) + schur + _vcycle_bytes(hu, s, precision == 1)
    op = 27 * 9 * 8 * nN + 2 * 24 * 8 * nT + 11 * 8 * nF + 17 * 8 * nT + 16 * n
    # the Arnoldi step's operator: FP64, or float-float words (8 B per
    # coefficient on A_uu's symmetric half) from the FP32 z
    op_arn = op if precision != 1 else 8 * (126 * nN + 64 * nT + 11 * nF) + 12 * n
    total = 16.0 * n  # right-hand side (reads the previous state, writes b)
    k = 0
    while k < iters_per_step:
        steps = min(m, iters_per_step - k)
        total += op + 16 * n            # residual of the cycle and its norm
        for j in range(steps):
            total += prec + op_arn + (2 * (j + 1) + 4) * 8 * n
        total += (steps + 2) * 8 * n    # x += Z y
        k += steps
    total += op + 16 * n                # true residual at exit
    return total


# ------------------------------------------------------------------ ranks
def reduce_max(value, dist, device):
    """Max of a per-rank float over all ranks (the job's time is its slowest
    rank's); identity on one process."""
    import torch
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_time(ms_max, world):
    """Whole-job time per step for a time-like metric with independent
    replicas: world systems advance one step in the slowest rank's time."""
    return ms_max / world


# ------------------------------------------------------------------ ours
def _timed_steps(s, args, world, dist, torch, launch_count, sample_clocks, local, kernel_timing=False):
    """W warm-up steps, then K timed steps of a fresh simulation (CUDA events
    on the library's stream), with clock sampling.  With kernel_timing the
    library also brackets every launch of its kernel classes with events
    (each Arnoldi step is then a host-driven graph replay, because event
    nodes cannot sit inside the conditional nodes of the whole-solve graph)."""
    x = None
    for _ in range(args.warmup):
        b = s.build_rhs(x)
        x, _ = s.solve(b, tol=TOL)
    x = None
    iters = []
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks_start(local) if sample_clocks else (None, None)
    if sample_clocks:
        time.sleep(0.3)
    l0 = launch_count()
    if kernel_timing:
        s.timing(True)
    e0.record(stream)
    for _ in range(args.steps):
        b = s.build_rhs(x)
        x, st = s.solve(b, tol=TOL)
        iters.append(st["iterations"])
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = launch_count() - l0
    ms = e0.elapsed_time(e1) / args.steps
    clocks = clocks_stop(*clk) if sample_clocks else None
    kt = s.timing_read(0) if kernel_timing else None
    if kernel_timing:
        s.timing(False)
    if world > 1:
        ms = reduce_max(ms, dist, "cuda")
    return dict(ms=ms, iters=iters, launches=launches, clocks=clocks, kt=kt)


def _solver(prob, precision, torch, restart=50, reorth=1, coarse_max=125, cheb_degree=2):
    from paper_2002_09603_gb300 import Solver, default_options
    opt = default_options()
    opt.precision = precision
    opt.restart = restart
    opt.reorth = reorth
    opt.coarse_max = coarse_max
    opt.cheb_degree = cheb_degree
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s = Solver(prob)
    s.assemble_condense()
    s.setup_precond(opt)
    e1.record(stream)
    torch.cuda.synchronize()
    return s, e0.elapsed_time(e1)


def _measure_workload(args, name, world, dist, torch, launch_count, local, precisions):
    """Both forms of one workload: FP64 plain, then mixed (the headline),
    each with its timed pass and a second pass with the kernel events on."""
    prob = make_problem(name)
    restart = args.restart if name == args.workload else WORKLOADS[name].get("restart", 12)
    out = {}
    for precision in precisions:
        s, setup = _solver(prob, precision, torch, restart, args.reorth, args.coarse_max, args.cheb_degree)
        r = _timed_steps(s, args, world, dist, torch, launch_count, precision == precisions[-1], local)
        rk = _timed_steps(s, args, world, dist, torch, launch_count, False, local, True)
        r["kt"], r["kernel_pass_ms"], r["setup_ms"] = rk["kt"], rk["ms"], setup
        r["op"] = s.timing_read(1)
        r["op_ff"] = s.timing_read(6)
        r["split"] = per_iteration_split(s, sum(rk["iters"]))
        r["hu"], r["hpi"] = s.hierarchy(0)["points"], s.hierarchy(1)["points"]
        r["cheb_degree"] = s.hierarchy(0)["cheb_degree"]
        r["restart"] = restart
        out[precision] = (s, r)
        if precision != precisions[-1]:
            s.close()
    return out


# the library's timing classes (mhfp_timing): what each costs per FGMRES
# iteration in the kernel-event pass
TIMING_SPLIT = {"preconditioner": 3, "displacement_vcycle": 4, "interface_pressure_vcycle": 5,
                "operator_arnoldi_ff": 6, "gram_schmidt": 2, "finest_sweeps": 0}


def per_iteration_split(s, iterations):
    """Microseconds per FGMRES iteration of each timing class (CUDA events
    around the library's launches), from the pass with kernel timing on."""
    out = {k: s.timing_read(c)["total_ms"] * 1e3 / max(iterations, 1) for k, c in TIMING_SPLIT.items()}
    out["note"] = ("us per iteration from the kernel-event pass (each Arnoldi step a host-driven graph replay "
                   "with event nodes); classes nest: the preconditioner holds both V-cycles")
    return out


def _sweep_roofline(kt, peak):
    avg_ms = kt["total_ms"] / max(kt["launches"], 1)
    gbs = kt["bytes_per_launch"] / (avg_ms * 1e-3) / 1e9 if kt["launches"] else None
    return avg_ms, gbs


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_2002_09603_gb300 import launch_count

    n_mesh = WORKLOADS[args.workload]["n"]
    peak, peak_kind = measured_peaks()
    precisions = {"both": (0, 1), "mixed": (1,), "fp64": (0,)}[args.precision]
    res = _measure_workload(args, args.workload, world, dist, torch, launch_count, local, precisions)
    s, r32 = res[precisions[-1]]
    r64 = res[0][1] if 0 in res else None
    ms = r32["ms"]
    setup_ms = r32["setup_ms"]

    # end to end through the C ABI with host buffers: the previous state comes
    # from pinned host memory and the solution goes back to it every step
    e2e = None
    if not args.no_e2e:
        nU, nP, _ = s.sizes
        h_state = torch.zeros(s.n, dtype=torch.float64).pin_memory()
        d_prev = s.empty()
        h2d = (nU + nP) * 8
        d2h = s.n * 8
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            d_prev[:nU + nP].copy_(h_state[:nU + nP], non_blocking=True)
            b = s.build_rhs(d_prev if k > 0 else None)
            xs, _ = s.solve(b, tol=TOL)
            h_state.copy_(xs, non_blocking=True)
            torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        if world > 1:
            e2e_ms = reduce_max(e2e_ms, dist, "cuda")
        e2e = {"value": aggregate_time(e2e_ms, world), "unit": "ms", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # roofline of the dominant sweep of the headline form
    headline_mixed = precisions[-1] == 1
    kname = "k_cheb_u0_sym<float>" if headline_mixed else "k_cheb_u0<double>"
    avg_ms, gbs = _sweep_roofline(r32["kt"], peak)
    roofline = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                "frac": gbs / peak if gbs else None,
                "traffic": traffic_for(kname, args.workload, r32["kt"]["bytes_per_launch"]),
                "kernel": (kname + " (Chebyshev sweep, finest displacement level, 27-point 3x3-block stencil"
                           + (", FP32, symmetric storage: 14 of the 27 blocks per node)" if headline_mixed
                              else ", FP64)")),
                "launches": r32["kt"]["launches"], "avg_launch_us": avg_ms * 1e3,
                "bytes_per_launch": r32["kt"]["bytes_per_launch"],
                "measured_in": "a second timed pass over the same K steps with the library's kernel events on "
                               f"(per-step graph replays, {r32.get('kernel_pass_ms', float('nan')):.2f} ms/step); the "
                               "headline pass runs each solve as one device-driven graph, which cannot hold event nodes",
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s"}
    # the FP64 operator A_H x (every apply of the FP64 form; the stopping
    # test of the mixed one) is bound by the FP64 pipe
    sm_max = ((r32["clocks"] or {}).get("sm_max_mhz") or 2070.0)
    fpk = fp64_peak_tflops(sm_max)
    r_op = r64 if r64 is not None else r32
    op = r_op["op"]
    op_ms = op["total_ms"] / max(op["launches"], 1)
    op_tf = operator_flops(n_mesh) / (op_ms * 1e-3) / 1e12 if op["launches"] and op_ms > 0 else None
    roofline_fp64 = {"bound": "alu", "achieved": op_tf, "peak": fpk, "unit": "TFLOP/s",
                     "frac": op_tf / fpk if op_tf else None, "traffic": None,
                     "kernel": "operator A_H x (k_apply_u + k_apply_p + k_apply_pi, FP64"
                               + (", FP64 form's run)" if r_op is not r32 else ")"),
                     "launches": op["launches"], "avg_launch_us": op_ms * 1e3,
                     "flops_per_launch": operator_flops(n_mesh),
                     "hbm_achieved_gbs": op["bytes_per_launch"] / (op_ms * 1e-3) / 1e9 if op_tf else None,
                     "peak_source": "derived FP64 pipe peak: 152 SMs x 2 FMA/clk x 2 flop x max SM clock"}
    # the mixed form's Arnoldi operator: float-float words, off the FP64
    # pipe, bound by HBM
    roofline_ff = None
    off = r32.get("op_ff") or {}
    if headline_mixed and off.get("launches") and off.get("total_ms", 0) > 0:
        ff_ms = off["total_ms"] / off["launches"]
        ff_gbs = off["bytes_per_launch"] / (ff_ms * 1e-3) / 1e9
        roofline_ff = {"bound": "hbm", "achieved": ff_gbs, "peak": peak, "unit": "GB/s", "frac": ff_gbs / peak,
                       "traffic": traffic_for("ff_operator", args.workload, off["bytes_per_launch"]),
                       "kernel": "Arnoldi operator A_H z in float-float (k_apply_u_ff + k_apply_p_ff + k_apply_pi_ff)",
                       "launches": off["launches"], "avg_launch_us": ff_ms * 1e3,
                       "bytes_per_launch": off["bytes_per_launch"],
                       "fp64_equivalent_tflops": operator_flops(n_mesh) / (ff_ms * 1e-3) / 1e12,
                       "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                       else "fallback 6.8 TB/s"}
    # the whole step against the bandwidth roofline
    mean_iters = statistics.mean(r32["iters"])
    sb = step_bytes(n_mesh, r32["hu"], r32["hpi"], precisions[-1], r32["restart"], int(round(mean_iters)))
    step_roof = {"bytes_per_step": sb, "achieved_gbs": sb / (ms * 1e-3) / 1e9, "peak": peak,
                 "frac": sb / (ms * 1e-3) / 1e9 / peak,
                 "model": "algorithmic bytes of every kernel of the step (bench.step_bytes), FP64 coarsest "
                          "inverse and L2-resident coarse levels included"}

    fp64_plain = None
    if r64 is not None and r64 is not r32:
        a64, g64 = _sweep_roofline(r64["kt"], peak)
        t64 = cheb_u0_flops(n_mesh) / (a64 * 1e-3) / 1e12 if r64["kt"]["launches"] else None
        sb64 = step_bytes(n_mesh, r64["hu"], r64["hpi"], 0, r64["restart"], int(round(statistics.mean(r64["iters"]))))
        fp64_plain = {"ms_per_step": r64["ms"], "iterations_per_step": r64["iters"], "setup_ms": r64["setup_ms"],
                      "gpu_launches": r64["launches"], "cheb_degree": r64["cheb_degree"],
                      "sweep_roofline": {"kernel": "k_cheb_u0<double>", "bound": "alu", "achieved": t64, "peak": fpk,
                                         "unit": "TFLOP/s", "frac": t64 / fpk if t64 else None,
                                         "hbm_achieved_gbs": g64, "avg_launch_us": a64 * 1e3},
                      "step_frac_of_hbm": sb64 / (r64["ms"] * 1e-3) / 1e9 / peak}

    # the 64^3 log-normal workload, measured in the same run
    other = None
    if args.workload == "layered128" and world == 1 and not args.no_64:
        o = _measure_workload(args, "lognormal64", world, dist, torch, launch_count, local, precisions)
        so, ro = o[precisions[-1]]
        ao, go = _sweep_roofline(ro["kt"], peak)
        other = {"workload": WORKLOADS["lognormal64"]["desc"], "unknowns": so.n, "restart": ro["restart"],
                 "ms_per_step": ro["ms"], "iterations_per_step": ro["iters"], "setup_ms": ro["setup_ms"],
                 "cheb_degree": ro["cheb_degree"],
                 "per_iteration_us": ro["split"],
                 "sweep_frac_of_hbm": go / peak if go else None,
                 "step_frac_of_hbm": step_bytes(64, ro["hu"], ro["hpi"], precisions[-1], ro["restart"],
                                                int(round(statistics.mean(ro["iters"])))) / (ro["ms"] * 1e-3) / 1e9 / peak,
                 "fp64_plain_ms_per_step": o[0][1]["ms"] if 0 in o and len(precisions) > 1 else None}
        so.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg(args.workload, mean_iters)

    nU, nP, nPi = s.sizes
    auu_mb = 27 * 9 * 8 * (n_mesh + 1) ** 3 / 1e6  # 27 3x3 FP64 blocks per node
    if rank == 0:
        line = {
            "metric": METRIC, "value": aggregate_time(ms, world), "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None,
            "dtype": ("f64 (FGMRES basis, Gram-Schmidt, stopping test and restarts) + float-float (Arnoldi operator, "
                      "48-bit significands) + f32 (V-cycles, Schur steps)" if headline_mixed else "f64"),
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"], "unknowns": s.n, "n_u": nU, "n_p": nP,
                       "n_pi": nPi, "tol": TOL, "restart": args.restart, "reorth": args.reorth,
                       "coarse_max": args.coarse_max, "iterations_per_step": r32["iters"],
                       "cheb_degree": r32["cheb_degree"],
                       "cheb_degree_source": "set-up autotuner" if args.cheb_degree == 0 else "option",
                       "setup_ms": setup_ms, "precision": {"both": "FP32 V-cycles inside FP64 FGMRES",
                                                           "mixed": "FP32 V-cycles inside FP64 FGMRES",
                                                           "fp64": "FP64 throughout"}[args.precision],
                       "fp64_plain": fp64_plain,
                       "l2": (f"inputs larger than L2 (A_uu alone is {auu_mb:.0f} MB in FP64, "
                              f"{auu_mb * 14 / 27 / 2:.0f} MB as the symmetric FP32 half)"),
                       "parallelism": "replicas",
                       "hierarchy_u": r32["hu"], "hierarchy_pi": r32["hpi"],
                       "per_iteration_us": r32["split"],
                       "lognormal64": other},
            "roofline": roofline, "roofline_fp64": roofline_fp64, "roofline_operator_ff": roofline_ff,
            "step_roofline": step_roof,
            "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": r32["launches"], "clocks": r32["clocks"],
        }
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()


def run_adjoint(args):
    """Auxiliary workload: one evaluation of J and its gradient with respect
    to the per-cell log-permeability (forward sweep, checkpointed reverse
    sweep with adjoint solves), on one handle whose permeability is updated
    in place (mhfp_update_logk) for every evaluation."""
    import numpy as np
    import torch
    import mhfp_inputs as mi
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_09603_gb300 import Solver, launch_count
    from paper_2002_09603_gb300.adjoint import MisfitGradient
    n, nsteps = 48, 10
    prob = mi.lognormal_cube(n, seed=5, sigma=1.0, dt=0.1)
    q = mi.lognormal_cube(n, seed=55, sigma=1.0, dt=0.1)
    s = Solver(q)
    s.assemble_condense()
    s.setup_precond()
    nU, nP, _ = s.sizes
    nodes = np.arange((n + 1) ** 3)
    top = nodes[nodes // ((n + 1) ** 2) == n]
    x, uz, pp = None, [], []
    for _ in range(nsteps):
        x, _ = s.solve(s.build_rhs(x), tol=1e-13)
        xc = x.cpu().numpy()
        uz.append(xc[3 * top + 2])
        pp.append(xc[nU:nU + nP])
    s.close()
    mg = MisfitGradient(prob, nsteps, uz, pp, tol=1e-10, checkpoint_every=3, precision=1, restart=20)
    logk = np.log(prob.kappa[:, 0])
    rng = np.random.default_rng(6)
    t0 = time.perf_counter()
    mg.value_and_grad(logk)  # creates and sets up the handle once
    torch.cuda.synchronize()
    first = time.perf_counter() - t0
    times = []
    l0 = launch_count()
    for k in range(max(1, args.steps)):
        lk = logk + 0.1 * rng.standard_normal(logk.shape)
        mg.stats = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J, g = mg.value_and_grad(lk)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    solves = len(mg.stats)
    line = {"metric": "time per J + dJ/d ln kappa evaluation (adjoint)", "value": statistics.mean(times) * 1e3,
            "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": 1, "ms_per_step": statistics.mean(times) * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (FGMRES, operator, Gram-Schmidt) + f32 (V-cycles, Schur steps)", "data": "synthetic",
            "config": {"workload": WORKLOADS["adjoint48"]["desc"], "cells": int(prob.n_cells), "steps": nsteps,
                       "checkpoint_every": 3, "solves_per_evaluation": solves,
                       "iterations_per_solve_min_max": [min(st["iterations"] for st in mg.stats),
                                                        max(st["iterations"] for st in mg.stats)],
                       "first_evaluation_ms_with_setup": first * 1e3,
                       "parameter_update": "mhfp_update_logk on one handle (no re-creation)"},
            "gpu_launches": (launch_count() - l0) // max(1, args.steps)}
    print(json.dumps(line), flush=True)
    mg.close()


def run_batch(args):
    """Auxiliary workload: many uneven instances x 4 loads; reports the time
    per solved system with every instance and load in one graph launch, the
    four loads of an instance in lockstep (the line's value), beside the same
    graph with the loads one after another, per-load batched calls and the
    solves one after another."""
    import torch
    import mhfp_inputs as mi
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_09603_gb300 import launch_count
    from paper_2002_09603_gb300.batch import prepare_batch, solve_loads

    probs = mi.batch_instances()
    t0 = time.perf_counter()
    # the headline's solver options: the coarsening limit and the set-up
    # autotuner's Chebyshev degree (chosen per instance)
    solvers = prepare_batch(probs, precision=1, restart=args.restart, reorth=args.reorth,
                            cheb_degree=args.cheb_degree, coarse_max=args.coarse_max)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    degrees = [sv.hierarchy(0)["cheb_degree"] for sv in solvers]
    for _ in range(max(1, args.warmup)):
        solve_loads(solvers, (1.0,))
    torch.cuda.synchronize()
    l0 = launch_count()
    t0 = time.perf_counter()
    res = solve_loads(solvers, mi.LOAD_SCALES)
    torch.cuda.synchronize()
    batched = time.perf_counter() - t0
    launches = launch_count() - l0
    nsys = len(solvers) * len(mi.LOAD_SCALES)
    ok = all(c == 0 for _, _, codes in res for c in codes)
    iters = [st["iterations"] for _, stats, _ in res for st in stats]
    # every instance x every load in one CUDA graph launch
    from paper_2002_09603_gb300.batch import LoadBatch
    t0 = time.perf_counter()
    lb = LoadBatch(solvers, mi.LOAD_SCALES, tol=TOL)
    torch.cuda.synchronize()
    graph_build_s = time.perf_counter() - t0
    lb.run()  # warm-up
    torch.cuda.synchronize()
    l1 = launch_count()
    t0 = time.perf_counter()
    _, gstats, gcodes = lb.run()
    one_launch = time.perf_counter() - t0
    one_launch_kernels = launch_count() - l1
    gok = all(c == 0 for c in gcodes)
    lb.close()
    # the same graph with each instance's four loads in lockstep: every
    # kernel of the solve launched once for the four right-hand sides
    t0 = time.perf_counter()
    lk = LoadBatch(solvers, mi.LOAD_SCALES, tol=TOL, lanes=len(mi.LOAD_SCALES))
    torch.cuda.synchronize()
    lock_build_s = time.perf_counter() - t0
    lk.run()  # warm-up
    torch.cuda.synchronize()
    l2 = launch_count()
    t0 = time.perf_counter()
    _, kstats, kcodes = lk.run()
    lockstep = time.perf_counter() - t0
    lockstep_kernels = launch_count() - l2
    kok = all(c == 0 for c in kcodes)
    lk.close()
    # the same solves one handle at a time
    t0 = time.perf_counter()
    for scale in mi.LOAD_SCALES:
        for sv in solvers:
            b = sv.build_rhs(None, load_scale=scale)
            sv.solve(b, tol=TOL)
            sv.stream.synchronize()
    serial = time.perf_counter() - t0
    unknowns = sum(sum(sv.sizes) for sv in solvers)
    line = {"metric": "time per solved system, batched (" + METRIC + ")", "value": lockstep * 1e3 / nsys, "unit": "ms",
            "n_gpus": 1, "steps": 1, "warmup": args.warmup, "ms_per_step": lockstep * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (FGMRES, operator, Gram-Schmidt) + f32 (V-cycles, Schur steps)", "data": "synthetic",
            "config": {"workload": WORKLOADS["batch48"]["desc"], "instances": len(solvers), "systems": nsys,
                       "restart": args.restart, "reorth": args.reorth, "coarse_max": args.coarse_max,
                       "cheb_degree": ("set-up autotuner, per instance: " if args.cheb_degree == 0 else "option: ")
                       + ", ".join(f"{d} x{degrees.count(d)}" for d in sorted(set(degrees))),
                       "unknowns_per_load": unknowns, "sizes": [p.nx for p in probs], "all_converged": ok,
                       "iterations_min_max": [min(iters), max(iters)], "setup_s": setup_s,
                       "serial_ms_per_system": serial * 1e3 / nsys,
                       "form": "one graph launch, each instance's loads in lockstep (mhfp_batch_create_lanes)",
                       "lockstep": {"ms_per_system": lockstep * 1e3 / nsys, "all_converged": kok,
                                    "graph_build_s": lock_build_s, "kernels": lockstep_kernels,
                                    "iterations_min_max": [min(st["iterations"] for st in kstats),
                                                           max(st["iterations"] for st in kstats)]},
                       "one_launch": {"ms_per_system": one_launch * 1e3 / nsys, "all_converged": gok,
                                      "graph_build_s": graph_build_s, "kernels": one_launch_kernels,
                                      "iterations_min_max": [min(st["iterations"] for st in gstats),
                                                             max(st["iterations"] for st in gstats)]},
                       "per_load_calls": {"ms_per_system": batched * 1e3 / nsys, "all_converged": ok,
                                          "iterations_min_max": [min(iters), max(iters)], "kernels": launches},
                       "speedup_one_launch_vs_serial": serial / one_launch,
                       "speedup_lockstep_vs_one_launch": one_launch / lockstep},
            "gpu_launches": lockstep_kernels}
    print(json.dumps(line), flush=True)
    for sv in solvers:
        sv.close()


def run_table(args):
    """Auxiliary workload, the comparison of Section 5 (Table tab:can_3): the
    cantilever at the paper's two finest single-GPU grids and both time
    steps, solved with the mixed formulation's M_II^(m) and the hybrid
    formulation's M_II^(h) and M_III^(h): FGMRES iterations, set-up time
    T_p, solve time T_s (CUDA events around the library calls; the first
    solve of each set-up is a warm-up)."""
    import torch
    import mhfp_inputs as mi
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_09603_gb300 import Solver, default_options, launch_count
    variants = [("M_II^(m)", 1, 0), ("M_II^(h)", 0, 0), ("M_III^(h)", 0, 1)]
    # Table tab:can_3: iterations and T_t [s] per preconditioner, for context
    paper = {(64, 0.1): ([55, 53, 36], [3.9, 3.5, 8.2], 36), (64, 1e-5): ([56, 52, 31], [4.2, 3.7, 7.7], 36),
             (128, 0.1): ([63, 63, 47], [5.7, 5.2, 10.7], 288), (128, 1e-5): ([71, 63, 43], [6.6, 5.6, 9.9], 288),
             (256, 0.1): ([90, 86, 63], [11.1, 9.9, 16.8], 2268),
             (256, 1e-5): ([95, 83, 59], [15.1, 10.1, 16.0], 2268)}
    grids = [int(g) for g in args.can3_grids.split(",") if g]
    restart = 30
    rows = []
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    l0 = launch_count()
    for n in grids:
        for dt in (0.1, 1e-5):
            prob = mi.cantilever_cube(n, dt=dt)
            for vi, (label, form, nk) in enumerate(variants):
                opt = default_options()
                opt.formulation, opt.near_kernel, opt.restart = form, nk, restart
                torch.cuda.synchronize()
                ev[0].record(stream)
                s = Solver(prob)
                s.assemble_condense()
                s.setup_precond(opt)
                ev[1].record(stream)
                b = s.build_rhs()
                x, st = s.solve(b, tol=1e-6)
                ts = []
                for _ in range(max(1, args.steps)):
                    ev[2].record(stream)
                    x, st = s.solve(b, tol=1e-6, out=x)
                    ev[3].record(stream)
                    torch.cuda.synchronize()
                    ts.append(ev[2].elapsed_time(ev[3]))
                pr = paper.get((n, dt))
                rows.append({"inv_h": n, "dofs": s.n, "dt": dt, "preconditioner": label,
                             "iterations": st["iterations"], "converged": bool(st["converged"]),
                             "T_p_ms": ev[0].elapsed_time(ev[1]), "T_s_ms": statistics.median(ts),
                             "T_t_ms": ev[0].elapsed_time(ev[1]) + statistics.median(ts),
                             "paper_iterations": pr[0][vi] if pr else None, "paper_T_t_s": pr[1][vi] if pr else None,
                             "paper_processes": pr[2] if pr else None})
                s.close()
                del x, b
                torch.cuda.empty_cache()
    top = max(grids)
    main_ts = [r["T_t_ms"] for r in rows if r["inv_h"] == top and r["preconditioner"] == "M_II^(h)"]
    line = {"metric": f"T_t (set-up + solve), Test 2 cantilever 1/h={top}, M_II^(h) (mean of both dt)",
            "value": statistics.mean(main_ts), "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": 1,
            "ms_per_step": statistics.mean(main_ts), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS["cantilever_can3"]["desc"], "restart": restart, "rows": rows},
            "gpu_launches": launch_count() - l0}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == "cantilever_can3":
        run_table(args)
        return
    if args.workload == "batch48":
        run_batch(args)
        return
    if args.workload == "adjoint48":
        run_adjoint(args)
        return
    if args.impl == "reference":
        os.environ.update(SINGLE_THREAD_ENV)  # before numpy is imported
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
