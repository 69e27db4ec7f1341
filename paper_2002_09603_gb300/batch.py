"""Many independent systems solved together (mhfp_solve_batch).

Marshalling only: one handle per instance, each on its own CUDA stream, so
the per-step CUDA-graph replays of different instances overlap on the
device; every right-hand side of a round is solved in one batched call.
"""
from __future__ import annotations

from ._lib import Solver, default_options, solve_batch


def prepare_batch(problems, precision=1, restart=12, autotune=1, reorth=1):
    import torch
    solvers = []
    for prob in problems:
        opt = default_options()
        opt.precision = precision
        opt.restart = restart
        opt.autotune = autotune
        opt.reorth = reorth
        st = torch.cuda.Stream()
        s = Solver(prob, stream=st)
        s.assemble_condense()
        s.setup_precond(opt)
        solvers.append(s)
    return solvers


def solve_loads(solvers, load_scales, tol=1e-8):
    """For each load scale, build every instance's right-hand side and solve
    all instances in one batched call.  Returns a list (per load) of
    (xs, stats, statuses)."""
    import torch
    out = []
    for scale in load_scales:
        rhs = [s.build_rhs(None, load_scale=scale) for s in solvers]
        for s in solvers:
            s.stream.synchronize()
        out.append(solve_batch(solvers, rhs, tol=tol))
    torch.cuda.synchronize()
    return out
