"""Flexible GMRES(m) with right preconditioning (oracle, FP64).

Section 5: GMRES with right preconditioning and zero initial guess, stopped
when the 2-norm of the residual falls below tau times the initial one.  The
flexible variant (stored preconditioned directions Z) is used so that the
preconditioner may vary between iterations.  Orthogonalisation is classical
Gram-Schmidt applied twice; the Hessenberg least-squares problem is reduced
by Givens rotations.  Reading: the iteration runs on the symmetrically
equilibrated system D_s A D_s y = D_s b (x = D_s y), and exits only when the
recomputed true residual also meets the tolerance (within 5%).
"""
from __future__ import annotations

import numpy as np


def fgmres(apply_A, apply_M, b, tol=1e-8, restart=50, maxit=1000, scale=None, x0=None):
    """Solve A x = b.  apply_M approximates A^-1.  With ``scale`` = D_s the
    iteration runs on the equilibrated system and norms are taken there.
    Returns (x, info) with info = dict(iters, resid_hist, converged, true_rel)."""
    n = b.shape[0]
    s = np.ones(n) if scale is None else scale
    x = np.zeros(n) if x0 is None else x0.copy()
    bs = s * b
    bnorm = np.linalg.norm(bs)
    hist = []
    if bnorm == 0.0:
        return np.zeros(n), dict(iters=0, resid_hist=[0.0], converged=True, true_rel=0.0)
    total = 0
    converged = False
    while total < maxit:
        r = s * (b - apply_A(x))
        beta = np.linalg.norm(r)
        if not hist:
            hist.append(beta / bnorm)
        if beta <= 1.05 * tol * bnorm:
            converged = True
            break
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(restart):
            Z[j] = apply_M(V[j] / s)                 # unscaled direction
            w = s * apply_A(Z[j])
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            h2 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h2
            H[:j + 1, j] = h + h2
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or total >= maxit:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Z[:k].T @ y
    true_rel = np.linalg.norm(s * (b - apply_A(x))) / bnorm
    converged = converged or true_rel <= 1.05 * tol
    return x, dict(iters=total, resid_hist=hist, converged=converged, true_rel=true_rel)
