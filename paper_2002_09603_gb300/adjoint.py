"""Gradient of a time-stepped misfit with respect to the per-cell
log-permeability, by the discrete adjoint, on the GPU.

Marshalling only: every step runs in libmhfp (mhfp_update_logk,
mhfp_build_rhs, mhfp_solve, mhfp_misfit, mhfp_adjoint_rhs,
mhfp_adjoint_solve, mhfp_grad_logk).  One handle is created and set up
once; each evaluation only updates its permeability in place.  The
forward sweep keeps every `checkpoint_every`-th state; the reverse sweep
recomputes each segment from its checkpoint, so device memory holds
N / k + k states instead of N.

    A x_n = f + C x_{n-1};   J = sum_n j_n(x_n)
    A^T lambda_n = grad j_n + C^T lambda_{n+1}
    dJ/d ln kappa_T = - sum_n lambda_n^T (dA/d ln kappa_T) x_n
"""
from __future__ import annotations

import numpy as np

from ._lib import Solver, default_options


def _with_logk(prob, logk):
    """Copy of `prob` whose diagonal permeability is exp(logk) per cell,
    keeping the anisotropy ratios of prob.kappa."""
    import mhfp_inputs as mi
    q = mi.Problem(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in prob.__dict__.items()})
    base = np.log(prob.kappa[:, 0])
    q.kappa = prob.kappa * np.exp(np.asarray(logk, float) - base)[:, None]
    return q


class MisfitGradient:
    """J(ln kappa) and dJ/d ln kappa for `nsteps` backward-Euler steps.

    uz_targets, p_targets: per-step target arrays (top-plane u_z per node,
    p per cell); the weights are 1/RMS^2 of the targets."""

    def __init__(self, prob, nsteps, uz_targets, p_targets, tol=1e-12, checkpoint_every=1, precision=0,
                 restart=50):
        import torch
        self.torch = torch
        self.prob = prob
        self.nsteps = int(nsteps)
        self.uz_t = [torch.as_tensor(np.asarray(t, float), device="cuda") for t in uz_targets]
        self.p_t = [torch.as_tensor(np.asarray(t, float), device="cuda") for t in p_targets]
        self.inv_su2 = 1.0 / float(np.mean(np.concatenate([np.asarray(t) for t in uz_targets]) ** 2))
        self.inv_sp2 = 1.0 / float(np.mean(np.concatenate([np.asarray(t) for t in p_targets]) ** 2))
        self.tol = tol
        self.k = max(1, int(checkpoint_every))
        self.precision = precision
        self.restart = restart
        self.stats = []

    def _solver(self, logk):
        """The handle, created and set up on the first call; every call sets
        its log-permeability (in place, mhfp_update_logk)."""
        if getattr(self, "_s", None) is None:
            opt = default_options()
            opt.precision = self.precision
            opt.restart = self.restart
            s = Solver(self.prob)
            s.assemble_condense()
            s.setup_precond(opt)
            self._s = s
        t = self.torch.as_tensor(np.ascontiguousarray(logk, dtype=np.float64), device=self._s.device)
        self._s.update_logk(t)
        return self._s

    def close(self):
        if getattr(self, "_s", None) is not None:
            self._s.close()
            self._s = None

    def _step(self, s, x_prev):
        b = s.build_rhs(x_prev)
        x, st = s.solve(b, tol=self.tol)
        self.stats.append(st)
        return x

    def value(self, logk):
        s = self._solver(logk)
        J = self.torch.zeros(1, dtype=self.torch.float64, device="cuda")
        g = s.empty()
        x = None
        for n in range(self.nsteps):
            x = self._step(s, x)
            s.misfit(x, self.uz_t[n], self.p_t[n], self.inv_su2, self.inv_sp2, J, g)
        return float(J.item())

    def value_and_grad(self, logk):
        torch = self.torch
        s = self._solver(logk)
        J = torch.zeros(1, dtype=torch.float64, device="cuda")
        g = s.empty()
        grad = torch.zeros(s.sizes[1], dtype=torch.float64, device="cuda")
        # forward sweep, keeping every k-th state (x_{-1} = 0 is implicit)
        ckpt = {}
        x = None
        for n in range(self.nsteps):
            if n % self.k == 0:
                ckpt[n] = None if x is None else x.clone()
            x = self._step(s, x)
        # reverse sweep, segment by segment
        lam_next = None
        starts = sorted(ckpt)
        for a in reversed(starts):
            b_end = min(a + self.k, self.nsteps)
            seg, xp = [], ckpt[a]
            for n in range(a, b_end):
                xp = self._step(s, xp)
                seg.append(xp)
            for n in range(b_end - 1, a - 1, -1):
                xn = seg[n - a]
                s.misfit(xn, self.uz_t[n], self.p_t[n], self.inv_su2, self.inv_sp2, J, g)
                rhs = s.adjoint_rhs(g, lam_next)
                lam, st = s.adjoint_solve(rhs, tol=self.tol)
                self.stats.append(st)
                s.grad_logk(lam, xn, grad)
                lam_next = lam
        Jv = float(J.item())
        return Jv, grad


def make_autograd(mg: MisfitGradient):
    """torch.autograd.Function wrapping J(ln kappa) with the adjoint gradient."""
    import torch

    class LogPermMisfit(torch.autograd.Function):
        @staticmethod
        def forward(ctx, logk):
            J, grad = mg.value_and_grad(logk.detach().cpu().numpy())
            ctx.save_for_backward(grad.to(logk.device, logk.dtype))
            return torch.tensor(J, dtype=logk.dtype, device=logk.device)

        @staticmethod
        def backward(ctx, gout):
            (grad,) = ctx.saved_tensors
            return gout * grad

    return LogPermMisfit.apply
