"""Discrete adjoint of the backward-Euler time stepping and the gradient of
a misfit with respect to the per-cell log-permeability (oracle, FP64).

Not in the paper: the forward model is its Section 2 system (Eq. stab_A,
hybrid form) stepped in time (Section 2.1), A x_n = f + C x_{n-1} with
C x = [0 ; A_pu u + S_eps|T| p ; 0].  For J = sum_n j_n(x_n):

    A^T lambda_n = grad j_n(x_n) + C^T lambda_{n+1},   lambda_{N+1} = 0
    dJ/dtheta    = - sum_n lambda_n^T (dA/dtheta) x_n      (f, C free of kappa)

theta_T = ln kappa_T scales the whole diagonal permeability of cell T, so
W_T = A_ww,T^-1 is proportional to kappa_T and dA/dtheta_T is cell T's
condensed flow contribution (Eq. hmfeSys).  TEST INFRASTRUCTURE ONLY.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import system


def top_uz_dofs(B):
    m = B.mesh
    nodes = np.arange(m.n_nodes)
    k = nodes // ((m.nx + 1) * (m.ny + 1))
    top = nodes[k == m.nz]
    return 3 * top + 2


class Misfit:
    """j_n(x) = 1/2 sum_top (u_z - u_z*)^2 / s_u^2 + 1/2 sum_cells (p - p*)^2 / s_p^2
    with per-step targets and s = RMS of the targets."""

    def __init__(self, B, uz_targets, p_targets):
        self.B = B
        self.dofs = top_uz_dofs(B)
        self.uz_t = [np.asarray(t, float) for t in uz_targets]
        self.p_t = [np.asarray(t, float) for t in p_targets]
        self.su2 = np.mean(np.concatenate(self.uz_t) ** 2)
        self.sp2 = np.mean(np.concatenate(self.p_t) ** 2)

    def value_and_grad(self, n, x):
        nU, nP, nPi = self.B.sizes
        du = x[self.dofs] - self.uz_t[n]
        dp = x[nU:nU + nP] - self.p_t[n]
        j = 0.5 * du @ du / self.su2 + 0.5 * dp @ dp / self.sp2
        g = np.zeros_like(x)
        g[self.dofs] = du / self.su2
        g[nU:nU + nP] = dp / self.sp2
        return j, g


def coupling_matrix(B):
    """C with b_n = f + C x_{n-1}."""
    nU, nP, nPi = B.sizes
    return sp.bmat([[sp.csr_matrix((nU, nU)), None, None],
                    [B.Apu, B.App, None],
                    [None, None, sp.csr_matrix((nPi, nPi))]], format="csr")


class _ScaledLU:
    """x = M^-1 b from an LU of D M D, D = |diag(M)|^(-1/2), plus two steps of
    iterative refinement (the blocks differ by many orders of magnitude)."""

    def __init__(self, M):
        self.M = M.tocsc()
        self.d = 1.0 / np.sqrt(np.abs(self.M.diagonal()))
        D = sp.diags(self.d)
        self.lu = spla.splu((D @ self.M @ D).tocsc())

    def solve(self, b):
        x = self.d * self.lu.solve(self.d * b)
        for _ in range(2):
            x = x + self.d * self.lu.solve(self.d * (b - self.M @ x))
        return x


def forward(B, nsteps, load_scale=1.0):
    A = system.system_matrix(B).tocsc()
    lu = _ScaledLU(A)
    nU, nP, _ = B.sizes
    xs, x = [], None
    for _ in range(nsteps):
        b = system.rhs(B, None if x is None else x[:nU], None if x is None else x[nU:nU + nP], load_scale)
        x = lu.solve(b)
        xs.append(x)
    return xs


def cell_derivative_apply(B, lam, x):
    """g_T = -lambda^T (dA/d ln kappa_T) x for all cells, from the condensed
    element blocks: p row dt (1^T W 1 p_T - (W 1)^T pi_T), pi rows
    W pi_T - W 1 p_T; drained faces are eliminated."""
    nU, nP, nPi = B.sizes
    W = np.linalg.inv(B.Aww_cells)
    W1 = W.sum(axis=2)
    s = W1.sum(axis=1)
    cf = B.mesh.cell_faces
    keep = (~B.pi_fixed)[cf].astype(float)
    p, lp = x[nU:nU + nP], lam[nU:nU + nP]
    pi_T = x[nU + nP:][cf] * keep
    lpi_T = lam[nU + nP:][cf] * keep
    prow = B.dt * (s * p - np.einsum("tf,tf->t", W1, pi_T))
    pirows = np.einsum("tfg,tg->tf", W, pi_T) - W1 * p[:, None]
    return -(lp * prow + np.einsum("tf,tf->t", lpi_T, pirows))


def gradient(B, nsteps, misfit, load_scale=1.0):
    """(J, dJ/d ln kappa) by the discrete adjoint with direct solves."""
    xs = forward(B, nsteps, load_scale)
    A = system.system_matrix(B)
    luT = _ScaledLU(A.T)
    C = coupling_matrix(B)
    J = 0.0
    grad = np.zeros(B.sizes[1])
    lam_next = None
    for n in range(nsteps - 1, -1, -1):
        j, g = misfit.value_and_grad(n, xs[n])
        J += j
        rhs = g if lam_next is None else g + C.T @ lam_next
        lam = luT.solve(rhs)
        grad += cell_derivative_apply(B, lam, xs[n])
        lam_next = lam
    return J, grad, xs


def objective(prob, nsteps, misfit_targets, load_scale=1.0):
    """J for a problem (fresh assembly), for finite differences."""
    B = system.assemble(prob)
    m = Misfit(B, *misfit_targets)
    xs = forward(B, nsteps, load_scale)
    return sum(m.value_and_grad(n, xs[n])[0] for n in range(nsteps))
