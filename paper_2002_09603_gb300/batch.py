"""Many independent systems solved together.

Marshalling only: one handle per instance.  `LoadBatch` binds
every (instance, load) pair into one CUDA graph (mhfp_batch_create) and
solves them all with one launch (mhfp_batch_run): the loads of an instance
run one after another in its branch, or, with lanes > 1, in lockstep
(mhfp_batch_create_lanes), the instances concurrently.
`solve_loads` is the earlier form: per load, one mhfp_solve_batch call that
launches each instance's solve graph on its own stream.
"""
from __future__ import annotations

from ._lib import Batch, Solver, default_options, solve_batch


def prepare_batch(problems, precision=1, restart=12, autotune=1, reorth=1, **options):
    """One set-up handle per problem, each on a stream of its own; `options`
    sets further mhfp_options fields by name."""
    import torch
    solvers = []
    for prob in problems:
        opt = default_options()
        opt.precision = precision
        opt.restart = restart
        opt.autotune = autotune
        opt.reorth = reorth
        for k, v in options.items():
            setattr(opt, k, v)
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


class LoadBatch:
    """Every instance x every load scale as one graph launch.  The right-hand
    sides are built once (mhfp_build_rhs); `run()` solves them all.  lanes > 1
    solves up to `lanes` loads of an instance in lockstep (each kernel once
    for all of them)."""

    def __init__(self, solvers, load_scales, tol=1e-8, lanes=1):
        import torch
        self.solvers = solvers
        self.scales = tuple(load_scales)
        entries, rhs, out = [], [], []
        for s in solvers:
            for scale in self.scales:
                entries.append(s)
                rhs.append(s.build_rhs(None, load_scale=scale))
                out.append(s.empty())
        for s in solvers:
            s.stream.synchronize()
        torch.cuda.synchronize()
        self.rhs, self.out = rhs, out
        self.batch = Batch(entries, rhs, out, tol=tol, lanes=lanes)

    def run(self, stream=None):
        """Returns (solutions, stats, statuses), entry order instance-major."""
        stats, codes = self.batch.run(stream)
        return self.out, stats, codes

    def close(self):
        self.batch.close()
