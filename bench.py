#!/usr/bin/env python3
"""Time-to-solve per backward-Euler step of the stabilized hybridized
poromechanics system (FGMRES + block-triangular multigrid preconditioner,
FP64) on one GB300, to a 1e-8 relative residual of the equilibrated system.

Default workload: 64^3 unit cube, log-normal permeability (ln kappa ~
N(ln 1e-13, 2^2), exponential covariance of 8 cells, seed 2), S_eps = 0,
dt = 1e-3 s, consolidation-column boundaries; 1,884,739 unknowns.  A "step"
is one time step: right-hand side from the previous state + FGMRES solve.
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

WORKLOADS = {
    "lognormal64": dict(n=64, restart=12, desc="64^3 hex, log-normal kappa (sigma 2, corr. 8 cells, seed 2), S_eps=0, dt=1e-3 s"),
    "lognormal32": dict(n=32, desc="32^3 hex, log-normal kappa (sigma 2, corr. 8 cells, seed 2), S_eps=0, dt=1e-3 s"),
    "lognormal96": dict(n=96, desc="96^3 hex, log-normal kappa (sigma 2, corr. 8 cells, seed 2), S_eps=0, dt=1e-3 s"),
    "layered128": dict(n=128, gen="layered", restart=20,
                       desc="128^3 hex, interior node jitter U(+-0.2h), 8 z-layers: kappa log-U[1e-18,1e-12] m^2, "
                            "E log-U[1e8,1e10] Pa, nu U[0.2,0.35]; S_eps=0, dt=0.1 s (seed 3)"),
    "batch48": dict(n=0, desc="48 cubes n ~ U{16..64} (seed 4), own log-normal kappa (sigma 1.5), loads x0.5/1/2/4, "
                              "FP32 V-cycles in FP64 FGMRES(12), one mhfp_solve_batch call per load"),
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
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="lognormal64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--restart", type=int, default=None,
                    help="FGMRES restart length (default: the fastest measured for the workload, 12 at 64^3, "
                         "20 at 128^3)")
    ap.add_argument("--coarse-max", type=int, default=512,
                    help="coarsen while a multigrid level has more lattice points (512: the 64^3 workload's "
                         "hierarchies end at 8^3 points, inverted densely on the GPU)")
    ap.add_argument("--reorth", type=int, choices=[0, 1], default=0,
                    help="Gram-Schmidt: 0 one classical pass (PETSc's GMRES default; same iterations and "
                         "residuals on the workloads), 1 DGKS reorthogonalisation when needed")
    ap.add_argument("--precision", choices=["both", "mixed", "fp64"], default="both",
                    help="both: mixed headline with FP64-plain beside it (default)")
    ap.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-target", type=str, default="", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.restart is None:
        args.restart = WORKLOADS[args.workload].get("restart", 12)
    return args


SINGLE_THREAD_ENV = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1",
                     "NUMEXPR_NUM_THREADS": "1"}


def oracle_sample_subprocess(workload, n_target_dofs, gpu_iters, sample_n=32):
    """Run the oracle sample in a fresh interpreter pinned to one BLAS/OpenMP
    thread (so the reported core count is exact), not forked from this
    CUDA process."""
    env = dict(os.environ, **SINGLE_THREAD_ENV)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--workload", workload,
                        "--oracle-sample", str(sample_n),
                        "--oracle-target", f"{n_target_dofs},{gpu_iters}"], env=env, capture_output=True,
                       text=True, timeout=600)
    if r.returncode != 0:
        return {"value": None, "unit": "ms", "cores": 1, "kind": "oracle", "sample": "failed: " + r.stderr[-300:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


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
def oracle_sample(workload, n_target_dofs, gpu_iters, sample_n=32, nsteps=1):
    """The FP64 oracle (as it stands) on a bounded sample of the workload:
    `nsteps` time steps of the same generator at sample_n^3 (setup not
    timed), scaled to the full workload by unknowns x FGMRES iterations."""
    import oracle
    from oracle import fgmres, precond, system
    prob = make_problem(workload, sample_n)
    B = oracle.assemble(prob)
    pc = precond.build(B, "amg")
    A = system.system_matrix(B)
    sc = precond.equilibration(B, pc.Bt, pc.C)
    nU, nP, _ = B.sizes
    n_s = sum(B.sizes)
    xprev = None
    secs, iters = [], []
    for _ in range(nsteps):
        t0 = time.perf_counter()
        b = system.rhs(B, None if xprev is None else xprev[:nU], None if xprev is None else xprev[nU:nU + nP])
        x, info = fgmres.fgmres(lambda v: A @ v, pc.apply, b, tol=TOL, scale=sc)
        secs.append(time.perf_counter() - t0)
        iters.append(info["iters"])
        xprev = x
    per_dof_iter = sum(secs) / (n_s * sum(iters))
    ms = per_dof_iter * n_target_dofs * gpu_iters * 1e3
    return dict(value=ms, unit="ms", cores=1, kind="oracle",
                sample=(f"{nsteps} time step(s) of the same workload generator at {sample_n}^3 ({n_s} unknowns, "
                        f"{sum(iters)} FGMRES iterations, {sum(secs):.2f} s, setup untimed) on one host core "
                        f"(scipy.sparse is single-threaded), scaled by unknowns x iterations to the full "
                        f"workload's {gpu_iters:.1f} iterations"),
                sample_seconds=sum(secs), sample_iters=iters), secs


def run_reference(args):
    """--impl reference: the oracle timed on the host cores, each step a
    bounded sample of the workload, scaled to the metric's unit."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_full = sum(make_problem_sizes(args.workload))
    import oracle
    from oracle import fgmres, precond, system
    sample_n = 24
    prob = make_problem(args.workload, sample_n)
    B = oracle.assemble(prob)
    pc = precond.build(B, "amg")
    A = system.system_matrix(B)
    sc = precond.equilibration(B, pc.Bt, pc.C)
    nU, nP, _ = B.sizes
    n_s = sum(B.sizes)
    xprev = None
    per_step = []
    total_iters = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        b = system.rhs(B, None if xprev is None else xprev[:nU], None if xprev is None else xprev[nU:nU + nP])
        x, info = fgmres.fgmres(lambda v: A @ v, pc.apply, b, tol=TOL, scale=sc)
        dt = time.perf_counter() - t0
        xprev = x
        if k >= args.warmup:
            per_step.append(dt * n_full / n_s * 1e3)
            total_iters.append(info["iters"])
    ms = sum(per_step) / len(per_step)
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"], "unknowns": n_full, "tol": TOL,
                       "parallelism": "replicas"},
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": 1, "kind": "oracle",
                             "sample": (f"each step = one time step of the same generator at {sample_n}^3 "
                                        f"({n_s} unknowns, {total_iters} FGMRES iterations), scaled by unknowns "
                                        f"to the full workload; one host core")},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def make_problem_sizes(name):
    n = WORKLOADS[name]["n"]
    return (3 * (n + 1) ** 3, n ** 3, 3 * n * n * (n + 1))


def traffic_for(kernel):
    """dram read+write bytes per launch of `kernel` at the 64^3 workload, from
    the committed ncu summary, or None if the kernel's source region changed
    since the counters were taken."""
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
    return d["bytes_per_launch"] if sha == d["region_sha"] else None


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


def _solver(prob, precision, torch, restart=50, reorth=1, coarse_max=125):
    from paper_2002_09603_gb300 import Solver, default_options
    opt = default_options()
    opt.precision = precision
    opt.restart = restart
    opt.reorth = reorth
    opt.coarse_max = coarse_max
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

    prob = make_problem(args.workload)
    n_mesh = WORKLOADS[args.workload]["n"]
    peak, peak_kind = measured_peaks()

    # FP64-plain form first (reported beside the headline), then the
    # mixed form (FP32 V-cycles and Schur steps inside FP64 FGMRES)
    r64, setup64 = None, None
    if args.precision in ("both", "fp64"):
        s64, setup64 = _solver(prob, 0, torch, args.restart, args.reorth, args.coarse_max)
        r64 = _timed_steps(s64, args, world, dist, torch, launch_count, args.precision == "fp64", local)
        r64["kt"] = _timed_steps(s64, args, world, dist, torch, launch_count, False, local, True)["kt"]
        if args.precision == "fp64":
            s, setup_ms, r32 = s64, setup64, r64
        else:
            s64.close()
            del s64
    if args.precision in ("both", "mixed"):
        s, setup_ms = _solver(prob, 1, torch, args.restart, args.reorth, args.coarse_max)
        r32 = _timed_steps(s, args, world, dist, torch, launch_count, True, local)
        # second pass over the same steps with the kernel events on (roofline)
        rk = _timed_steps(s, args, world, dist, torch, launch_count, False, local, True)
        r32["kt"] = rk["kt"]
        r32["kernel_pass_ms"] = rk["ms"]
    ms = r32["ms"]

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

    # roofline of the dominant sweep of the headline (mixed) form:
    # k_cheb_u0_sym<float>, HBM-bound
    kt = r32["kt"]
    avg_ms = kt["total_ms"] / max(kt["launches"], 1)
    gbs = kt["bytes_per_launch"] / (avg_ms * 1e-3) / 1e9 if kt["launches"] else None
    roofline = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                "frac": gbs / peak if gbs else None,
                "traffic": traffic_for("k_cheb_u0_sym<float>") if args.workload == "lognormal64" else None,
                "kernel": "k_cheb_u0_sym<float> (Chebyshev sweep, finest displacement level, 27-point 3x3-block "
                          "stencil, FP32, symmetric storage: 14 of the 27 blocks per node)",
                "launches": kt["launches"], "avg_launch_us": avg_ms * 1e3, "bytes_per_launch": kt["bytes_per_launch"],
                "measured_in": "a second timed pass over the same K steps with the library's kernel events on "
                               f"(per-step graph replays, {r32.get('kernel_pass_ms', float('nan')):.2f} ms/step); the "
                               "headline pass runs each solve as one device-driven graph, which cannot hold event nodes",
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s"}
    # the FP64-plain form's dominant kernel is bound by the FP64 pipe
    k64 = (r64 or r32)["kt"]
    avg64 = k64["total_ms"] / max(k64["launches"], 1)
    sm_max = ((r32["clocks"] or {}).get("sm_max_mhz") or 2070.0)
    fpk = fp64_peak_tflops(sm_max)
    tf64 = cheb_u0_flops(n_mesh) / (avg64 * 1e-3) / 1e12 if k64["launches"] else None
    roofline_fp64 = {"bound": "alu", "achieved": tf64, "peak": fpk, "unit": "TFLOP/s",
                     "frac": tf64 / fpk if tf64 else None,
                     "traffic": traffic_for("k_cheb_u0<double>") if args.workload == "lognormal64" else None,
                     "kernel": "k_cheb_u0<double>", "avg_launch_us": avg64 * 1e3,
                     "hbm_achieved_gbs": k64["bytes_per_launch"] / (avg64 * 1e-3) / 1e9 if k64["launches"] else None,
                     "peak_source": "derived FP64 pipe peak: 152 SMs x 2 FMA/clk x 2 flop x max SM clock"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample_subprocess(args.workload, s.n, statistics.mean(r32["iters"]))

    nU, nP, nPi = s.sizes
    auu_mb = 27 * 9 * 8 * (n_mesh + 1) ** 3 / 1e6  # 27 3x3 FP64 blocks per node
    if rank == 0:
        line = {
            "metric": METRIC, "value": aggregate_time(ms, world), "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (FGMRES, operator, Gram-Schmidt) + f32 (V-cycles, Schur steps)",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"], "unknowns": s.n, "n_u": nU, "n_p": nP,
                       "n_pi": nPi, "tol": TOL, "restart": args.restart, "reorth": args.reorth,
                       "coarse_max": args.coarse_max, "iterations_per_step": r32["iters"],
                       "setup_ms": setup_ms, "precision": {"both": "FP32 V-cycles inside FP64 FGMRES",
                                                           "mixed": "FP32 V-cycles inside FP64 FGMRES",
                                                           "fp64": "FP64 throughout"}[args.precision],
                       "fp64_plain": None if r64 is None else {
                           "ms_per_step": r64["ms"], "iterations_per_step": r64["iters"], "setup_ms": setup64,
                           "gpu_launches": r64["launches"]},
                       "l2": (f"inputs larger than L2 (A_uu alone is {auu_mb:.0f} MB in FP64, "
                              f"{auu_mb * 14 / 27 / 2:.0f} MB as the symmetric FP32 half)"),
                       "parallelism": "replicas",
                       "hierarchy_u": s.hierarchy(0)["points"], "hierarchy_pi": s.hierarchy(1)["points"]},
            "roofline": roofline, "roofline_fp64": roofline_fp64, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": r32["launches"], "clocks": r32["clocks"],
        }
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()


def run_batch(args):
    """Auxiliary workload: many uneven instances x 4 loads; reports the time
    per solved system with all instances batched (concurrent streams and
    graph replays) beside the same solves one after another."""
    import torch
    import mhfp_inputs as mi
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_09603_gb300 import launch_count
    from paper_2002_09603_gb300.batch import prepare_batch, solve_loads

    probs = mi.batch_instances()
    t0 = time.perf_counter()
    solvers = prepare_batch(probs, precision=1, restart=args.restart, reorth=args.reorth)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
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
    # the same solves one handle at a time
    t0 = time.perf_counter()
    for scale in mi.LOAD_SCALES:
        for sv in solvers:
            b = sv.build_rhs(None, load_scale=scale)
            sv.solve(b, tol=TOL)
            sv.stream.synchronize()
    serial = time.perf_counter() - t0
    unknowns = sum(sum(sv.sizes) for sv in solvers)
    line = {"metric": "time per solved system, batched (" + METRIC + ")", "value": batched * 1e3 / nsys, "unit": "ms",
            "n_gpus": 1, "steps": 1, "warmup": args.warmup, "ms_per_step": batched * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (FGMRES, operator, Gram-Schmidt) + f32 (V-cycles, Schur steps)", "data": "synthetic",
            "config": {"workload": WORKLOADS["batch48"]["desc"], "instances": len(solvers), "systems": nsys,
                       "restart": args.restart, "reorth": args.reorth,
                       "unknowns_per_load": unknowns, "sizes": [p.nx for p in probs], "all_converged": ok,
                       "iterations_min_max": [min(iters), max(iters)], "setup_s": setup_s,
                       "serial_ms_per_system": serial * 1e3 / nsys, "batched_speedup": serial / batched},
            "gpu_launches": launches}
    print(json.dumps(line), flush=True)
    for sv in solvers:
        sv.close()


def main():
    args = parse()
    if args.workload == "batch48":
        run_batch(args)
        return
    if args.oracle_sample:
        tgt, it = args.oracle_target.split(",")
        d, _ = oracle_sample(args.workload, int(tgt), float(it), sample_n=args.oracle_sample)
        print(json.dumps(d), flush=True)
        return
    if args.impl == "reference":
        os.environ.update(SINGLE_THREAD_ENV)  # before numpy is imported
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
