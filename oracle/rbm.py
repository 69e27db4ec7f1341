"""M_III^(h) of Section 5: the displacement block's multigrid takes the six
rigid-body modes as its near-kernel (the paper uses PETSc GAMG "with the near
kernel information provided by the rigid body modes"); the interface-
pressure block and the Schur steps are those of M_II^(h).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Parity unpinned by the
paper for the multigrid internals: GAMG is named, not defined.  This is the
textbook smoothed-aggregation construction with a vector near-kernel,
written out plainly:

* level 0: the nodes of the Q1 lattice, three dofs each; near-kernel N_0 =
  the six rigid-body modes (three translations, three rotations about the
  mesh centroid), with the rows of prescribed dofs zeroed;
* aggregates: 3x3x3 boxes of lattice points (as in the M_II^(h) spec);
* tentative prolongator: on each aggregate the thin QR factorisation of N
  restricted to the aggregate's dofs, N_K = Q_K R_K, by classical Gram-
  Schmidt applied twice in mode order (translations x, y, z, then rotations
  about x, y, z) with a non-negative diagonal of R_K; a mode whose norm
  after orthogonalisation is at most 1e-10 of its norm before (or zero) is
  one the aggregate cannot represent (prescribed displacements, or too few
  points, leave it fewer rigid motions): its column of Q_K is zero.  Q_K
  becomes the aggregate's block of P_t and R_K the coarse near-kernel of
  the coarse point K.  Every coarse point carries six dofs; a dof whose
  column is zero has no fine support and gets a unit diagonal on the
  coarse level, as the M_II^(h) spec does for a coarse dof with no free
  fine dof (reading: GAMG is named, not defined; without pivoting the
  factorisation is unique, and a fixed block size keeps the coarse levels
  lattice operators);
* P = (I - omega D^-1 A) P_t with D the point-block diagonal and
  omega = 4 / (3 lmax), lmax = 1.1 rho(D^-1 A) by 15 power iterations from
  the same start vector as M_II^(h);
* Galerkin coarse operators P^T A P; coarsen while a level has more than
  coarse_max lattice points; the last level is solved with its dense
  inverse; V(1,1) cycle with Chebyshev(2) smoothing preconditioned by the
  point-block diagonal on [lmax/10, lmax].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import precond

QR_DROP = 1e-10
NK = 6   # dofs per coarse point: the six rigid-body modes


def rigid_body_modes(coords: np.ndarray, free: np.ndarray | None = None) -> np.ndarray:
    """(3 n_nodes) x 6 matrix of the rigid-body displacements of the nodes:
    translations along x, y, z, then rotations about the x, y and z axes
    through the centroid of the nodes.  Rows of dofs with free == False are
    zero."""
    x = np.asarray(coords, float) - np.asarray(coords, float).mean(axis=0)
    n = x.shape[0]
    N = np.zeros((n, 3, 6))
    for a in range(3):
        N[:, a, a] = 1.0
    # rotation about x: (0, -z, y); about y: (z, 0, -x); about z: (-y, x, 0)
    N[:, 1, 3], N[:, 2, 3] = -x[:, 2], x[:, 1]
    N[:, 0, 4], N[:, 2, 4] = x[:, 2], -x[:, 0]
    N[:, 0, 5], N[:, 1, 5] = -x[:, 1], x[:, 0]
    N = N.reshape(3 * n, 6)
    if free is not None:
        N[~np.asarray(free, bool)] = 0.0
    return N


@dataclass
class RLevel:
    A: sp.csr_matrix
    pts: list                      # dof indices of each lattice point
    dims: tuple                    # lattice dims (points)
    Dm: sp.csr_matrix | None = None  # point-block-diagonal inverse
    lmax: float = 0.0
    Pt: sp.csr_matrix | None = None
    P: sp.csr_matrix | None = None
    dense_inv: np.ndarray | None = None


def point_block_inverse(A: sp.csr_matrix, pts) -> sp.csr_matrix:
    rows, cols, vals = [], [], []
    Ad = A.tocsr()
    for dofs in pts:
        if len(dofs) == 0:
            continue
        blk = Ad[dofs][:, dofs].toarray()
        inv = np.linalg.inv(blk)
        rr, cc = np.meshgrid(dofs, dofs, indexing="ij")
        rows.append(rr.ravel())
        cols.append(cc.ravel())
        vals.append(inv.ravel())
    n = A.shape[0]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def _finish(lev: RLevel):
    lev.Dm = point_block_inverse(lev.A, lev.pts)
    v = precond.power_start(lev.A.shape[0])
    v /= np.linalg.norm(v)
    rho = 0.0
    for _ in range(precond.POWER_ITERS):
        w = lev.Dm @ (lev.A @ v)
        rho = np.linalg.norm(w)
        v = w / rho
    lev.lmax = 1.1 * rho


def gram_schmidt_modes(NK: np.ndarray):
    """Thin QR of the aggregate's near-kernel block NK (rows x 6) by
    classical Gram-Schmidt applied twice, columns in mode order, R with a
    non-negative diagonal; a column left with at most QR_DROP of its norm is
    dropped (zero column of Q, zero row of R).  Returns Q, R, kept."""
    m, k = NK.shape
    Q = np.zeros((m, k))
    R = np.zeros((k, k))
    kept = np.zeros(k, bool)
    for j in range(k):
        v = NK[:, j].copy()
        n0 = np.linalg.norm(v)
        for _ in range(2):
            h = Q[:, :j].T @ v
            v -= Q[:, :j] @ h
            R[:j, j] += h
        nv = np.linalg.norm(v)
        if n0 > 0.0 and nv > QR_DROP * n0:
            Q[:, j] = v / nv
            R[j, j] = nv
            kept[j] = True
    return Q, R, kept


def _tentative(lev: RLevel, N: np.ndarray):
    """P_t, the coarse points' dof lists, the coarse near-kernel, the coarse
    dofs with fine support (kept modes) and the coarse lattice dims."""
    agg, cdims = precond.aggregate_map(lev.dims)
    nc_pts = cdims[0] * cdims[1] * cdims[2]
    members = [[] for _ in range(nc_pts)]
    for p, K in enumerate(agg):
        members[K].append(p)
    rows, cols, vals = [], [], []
    Nc = np.zeros((NK * nc_pts, NK))
    active = np.zeros(NK * nc_pts, bool)
    for K in range(nc_pts):
        dofs = np.concatenate([np.asarray(lev.pts[p], dtype=np.int64) for p in members[K]])
        Q, R, kept = gram_schmidt_modes(N[dofs])
        rr, cc = np.meshgrid(dofs, NK * K + np.arange(NK), indexing="ij")
        rows.append(rr.ravel())
        cols.append(cc.ravel())
        vals.append(Q.ravel())
        Nc[NK * K:NK * K + NK] = R
        active[NK * K:NK * K + NK] = kept
    Pt = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(lev.A.shape[0], NK * nc_pts))
    Pt.eliminate_zeros()
    cpts = [np.arange(NK * K, NK * K + NK) for K in range(nc_pts)]
    return Pt, cpts, Nc, active, cdims


def build_u_hierarchy(B, coarse_max=precond.COARSE_MAX):
    m = B.mesh
    dims = (m.nx + 1, m.ny + 1, m.nz + 1)
    pts = [np.arange(3 * p, 3 * p + 3) for p in range(m.n_nodes)]
    lev = RLevel(B.Auu.tocsr(), pts, dims)
    N = rigid_body_modes(m.coords, ~B.u_fixed)
    levels = [lev]
    while dims[0] * dims[1] * dims[2] > coarse_max:
        _finish(lev)
        Pt, cpts, Nc, active, dims = _tentative(lev, N)
        omega = 4.0 / (3.0 * lev.lmax)
        P = (Pt - omega * (lev.Dm @ (lev.A @ Pt))).tocsr()
        lev.Pt, lev.P = Pt, P
        Ac = (P.T @ lev.A @ P).tocsr()
        Ac = (0.5 * (Ac + Ac.T)).tocsr()  # exact in real arithmetic; removes rounding asymmetry
        Ac = (Ac + sp.diags(np.where(active, 0.0, 1.0))).tocsr()
        Ac.sum_duplicates()
        lev = RLevel(Ac, cpts, dims)
        N = Nc
        levels.append(lev)
    lev.dense_inv = np.linalg.inv(lev.A.toarray())
    return levels


def chebyshev(lev: RLevel, b, x, degree=precond.CHEB_DEGREE):
    lmax = lev.lmax
    lmin = lmax / precond.CHEB_RATIO
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = b - lev.A @ x
    d = (lev.Dm @ r) / theta
    x = x + d
    for _ in range(degree - 1):
        r = b - lev.A @ x
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (lev.Dm @ r)
        x = x + d
        rho = rho_new
    return x


def vcycle(levels, b, l=0):
    lev = levels[l]
    if lev.dense_inv is not None:
        return lev.dense_inv @ b
    x = chebyshev(lev, b, np.zeros_like(b))
    r = b - lev.A @ x
    xc = vcycle(levels, lev.P.T @ r, l + 1)
    x = x + lev.P @ xc
    return chebyshev(lev, b, x)
