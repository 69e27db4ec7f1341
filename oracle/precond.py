"""Block upper-triangular Schur-complement preconditioner (oracle, FP64).

Eq. (hybridPrec): M = [[A_uu, A_up, 0], [0, B~_p, dt A_ppi], [0, 0, C~_pi]],
applied by back substitution (pi, then p, then u; the explicit M^-1 is
given in the proof of Theorem 1).

Eq. (app_Bp) and the M_I^(h) definition in Section 5: B~_p = H~ + dt
diag(A_wp^T A_ww^-1 A_wp) with H~ = A_pp + diag(A_stab) + diag(A_up^T
diag(A_uu)^-1 A_up) (reading: the A_pp written for M_I^(h) is the storage
term, and the dt term is the one of Eq. (app_Bp)).
C~_pi = A_pipi - dt A_pip B~_p^-1 A_ppi (Section 4).

The paper's inner AMG solvers (PETSc GAMG, hypre) are not specified beyond
their names, so the multigrid here follows this library's own spec,
restated independently of the CUDA code:

* displacement block: smoothed aggregation on the node lattice, aggregates
  are 3x3x3 node boxes (i//3, j//3, k//3), tentative prolongator = aggregate
  indicator times I_3 (separate displacement components), restricted to
  free dofs; P = (I - omega D^-1 A) P_t with D the 3x3 node-block diagonal;
* interface-pressure block: faces -> cells by P_0[f,T] = 1/2 (interior face)
  or 1 (boundary face), 0 on drained faces; below the cell level the same
  smoothed aggregation as above, scalar;
* omega = 4 / (3 lmax), lmax = 1.1 * rho, rho from 15 power iterations on
  D^-1 A from v0[d] = 1 + ((7919 d) mod 97) / 97;
* Galerkin coarse operators P^T A P; a coarse dof with no free fine dof gets
  a unit diagonal;
* coarsen while a level has more than coarse_max lattice points (default
  125); exact dense solve
  on the last level;
* V(1,1) cycle, smoother = Chebyshev of degree 2 preconditioned by D on
  [lmax/10, lmax].

Parity with the CUDA path is at the level of the operators built here; the
paper itself pins none of these choices (parity unpinned by the paper for
the multigrid; it is pinned by convergence to the direct solution).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .system import Blocks

COARSE_MAX = 125
CHEB_DEGREE = 2
CHEB_RATIO = 10.0
POWER_ITERS = 15


def btilde(B: Blocks) -> np.ndarray:
    dAuu = B.Auu.diagonal()
    fixed_stress = np.asarray((B.Aup.multiply(B.Aup)).T @ (1.0 / dAuu)).ravel()
    return B.App.diagonal() + B.Astab.diagonal() + fixed_stress + B.dt * B.Dw


def ctilde(B: Blocks, Bt: np.ndarray) -> sp.csr_matrix:
    C = B.Apipi - B.dt * (B.Apip @ sp.diags(1.0 / Bt) @ B.Appi)
    C = C.tocsr()
    C.sum_duplicates()
    return C


def equilibration(B: Blocks, Bt, C) -> np.ndarray:
    """Symmetric diagonal scaling D_s = diag(A_uu, B~_p, C~_pi)^(-1/2) used by
    both sides so the stopping test sees every block (not in the paper)."""
    d = np.concatenate([B.Auu.diagonal(), Bt, C.diagonal()])
    return 1.0 / np.sqrt(d)


def power_start(n):
    d = np.arange(n, dtype=np.int64)
    return 1.0 + ((7919 * d) % 97).astype(np.float64) / 97.0


def block_diag_inv(A: sp.csr_matrix, bs: int):
    n = A.shape[0] // bs
    D = np.zeros((n, bs, bs))
    Acoo = A.tocoo()
    r, c, v = Acoo.row, Acoo.col, Acoo.data
    same = (r // bs) == (c // bs)
    np.add.at(D, (r[same] // bs, r[same] % bs, c[same] % bs), v[same])
    return np.linalg.inv(D)


def apply_block(Dinv, x, bs):
    n = Dinv.shape[0]
    return np.einsum("nij,nj->ni", Dinv, x.reshape(n, bs)).ravel()


def spectral_radius(A, Dinv, bs):
    v = power_start(A.shape[0])
    v /= np.linalg.norm(v)
    rho = 0.0
    for _ in range(POWER_ITERS):
        w = apply_block(Dinv, A @ v, bs)
        rho = np.linalg.norm(w)
        v = w / rho
    return rho


@dataclass
class Level:
    A: sp.csr_matrix
    bs: int
    dims: tuple | None           # lattice dims (points), None for the face level
    Dinv: np.ndarray | None = None
    lmax: float = 0.0
    P: sp.csr_matrix | None = None
    active: np.ndarray | None = None
    dense_inv: np.ndarray | None = None


def aggregate_map(dims):
    Lx, Ly, Lz = dims
    idx = np.arange(Lx * Ly * Lz)
    i, j, k = idx % Lx, (idx // Lx) % Ly, idx // (Lx * Ly)
    cd = (-(-Lx // 3), -(-Ly // 3), -(-Lz // 3))
    return (i // 3) + cd[0] * ((j // 3) + cd[1] * (k // 3)), cd


def _sa_prolongator(lev: Level):
    """Smoothed-aggregation prolongator of one lattice level."""
    bs = lev.bs
    agg, cdims = aggregate_map(lev.dims)
    nf = agg.shape[0]
    nc = cdims[0] * cdims[1] * cdims[2]
    rows = (bs * np.arange(nf)[:, None] + np.arange(bs)[None, :]).ravel()
    cols = (bs * agg[:, None] + np.arange(bs)[None, :]).ravel()
    vals = lev.active.astype(float)
    Pt = sp.csr_matrix((vals, (rows, cols)), shape=(bs * nf, bs * nc))
    Pt.eliminate_zeros()
    omega = 4.0 / (3.0 * lev.lmax)
    AP = (lev.A @ Pt).tocsr()
    DAP = _block_diag_matrix(lev.Dinv) @ AP
    P = (Pt - omega * DAP).tocsr()
    active_c = np.zeros(bs * nc, bool)
    active_c[cols[lev.active]] = True
    return P, cdims, active_c


def _block_diag_matrix(Dinv):
    return sp.block_diag([sp.csr_matrix(d) for d in Dinv], format="csr")


def _finish_level(lev: Level):
    lev.Dinv = block_diag_inv(lev.A, lev.bs)
    rho = spectral_radius(lev.A, lev.Dinv, lev.bs)
    lev.lmax = 1.1 * rho


def _galerkin(P, A, active_c):
    Ac = (P.T @ A @ P).tocsr()
    fix = np.where(active_c, 0.0, 1.0)
    Ac = (Ac + sp.diags(fix)).tocsr()
    Ac.sum_duplicates()
    return Ac


def _dense_coarse(lev: Level):
    lev.dense_inv = np.linalg.inv(lev.A.toarray())


def build_u_hierarchy(B: Blocks, coarse_max=COARSE_MAX):
    m = B.mesh
    dims = (m.nx + 1, m.ny + 1, m.nz + 1)
    lev = Level(B.Auu.tocsr(), 3, dims, active=~B.u_fixed)
    levels = [lev]
    while lev.dims[0] * lev.dims[1] * lev.dims[2] > coarse_max:
        _finish_level(lev)
        P, cdims, act = _sa_prolongator(lev)
        lev.P = P
        lev = Level(_galerkin(P, lev.A, act), 3, cdims, active=act)
        levels.append(lev)
    _dense_coarse(lev)
    return levels


def face_to_cell_prolongator(B: Blocks) -> sp.csr_matrix:
    m = B.mesh
    fc = m.face_cells
    ncell = (fc >= 0).sum(axis=1)
    w = np.where(ncell == 2, 0.5, 1.0) * (~B.pi_fixed)
    rows, cols, vals = [], [], []
    for s in range(2):
        has = fc[:, s] >= 0
        rows.append(np.flatnonzero(has))
        cols.append(fc[has, s])
        vals.append(w[has])
    P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(m.n_faces, m.n_cells))
    P.eliminate_zeros()
    return P


def build_pi_hierarchy(B: Blocks, C: sp.csr_matrix, coarse_max=COARSE_MAX):
    m = B.mesh
    lev = Level(C.tocsr(), 1, None, active=~B.pi_fixed)
    levels = [lev]
    if m.n_faces <= coarse_max:
        _dense_coarse(lev)
        return levels
    _finish_level(lev)
    P0 = face_to_cell_prolongator(B)
    lev.P = P0
    act = np.asarray(abs(P0).sum(axis=0)).ravel() > 0
    lev = Level(_galerkin(P0, lev.A, act), 1, (m.nx, m.ny, m.nz), active=act)
    levels.append(lev)
    while lev.dims[0] * lev.dims[1] * lev.dims[2] > coarse_max:
        _finish_level(lev)
        P, cdims, act = _sa_prolongator(lev)
        lev.P = P
        lev = Level(_galerkin(P, lev.A, act), 1, cdims, active=act)
        levels.append(lev)
    _dense_coarse(lev)
    return levels


def chebyshev(lev: Level, b, x, degree=CHEB_DEGREE):
    """Chebyshev iteration of the given degree for A x = b, preconditioned by
    the (block) diagonal, on the interval [lmax/ratio, lmax]."""
    lmax = lev.lmax
    lmin = lmax / CHEB_RATIO
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = b - lev.A @ x
    d = apply_block(lev.Dinv, r, lev.bs) / theta
    x = x + d
    for _ in range(degree - 1):
        r = b - lev.A @ x
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * apply_block(lev.Dinv, r, lev.bs)
        x = x + d
        rho = rho_new
    return x


def vcycle(levels, b, l=0, degree=CHEB_DEGREE):
    lev = levels[l]
    if lev.dense_inv is not None:
        return lev.dense_inv @ b
    x = chebyshev(lev, b, np.zeros_like(b), degree)
    r = b - lev.A @ x
    xc = vcycle(levels, lev.P.T @ r, l + 1, degree)
    x = x + lev.P @ xc
    return chebyshev(lev, b, x, degree)


@dataclass
class Preconditioner:
    B: Blocks
    Bt: np.ndarray
    C: sp.csr_matrix
    kind: str                      # "exact" (M_I), "amg" (M_II) or "amg_rbm" (M_III)
    u_levels: list = field(default_factory=list)
    pi_levels: list = field(default_factory=list)
    _luu: object = None
    _lpi: object = None

    def solve_uu(self, r):
        if self.kind == "exact":
            return self._luu.solve(r)
        if self.kind == "amg_rbm":
            from . import rbm
            return rbm.vcycle(self.u_levels, r)
        return vcycle(self.u_levels, r)

    def solve_pi(self, r):
        if self.kind == "exact":
            return self._lpi.solve(r)
        return vcycle(self.pi_levels, r)

    def apply(self, v):
        """Back substitution with M (Eq. hybridPrec): pi, then p, then u."""
        nU, nP, nPi = self.B.sizes
        vu, vp, vpi = v[:nU], v[nU:nU + nP], v[nU + nP:]
        zpi = self.solve_pi(vpi)
        zp = (vp - self.B.dt * (self.B.Appi @ zpi)) / self.Bt
        zu = self.solve_uu(vu - self.B.Aup @ zp)
        return np.concatenate([zu, zp, zpi])

    def apply_transpose(self, v):
        """Forward substitution with M^T = [[A_uu, 0, 0], [A_up^T, B~_p, 0],
        [0, dt A_ppi^T, C~_pi^T]] (u, then p, then pi); A_uu and C~_pi are
        symmetric and so are the V-cycles that stand for their inverses."""
        nU, nP, nPi = self.B.sizes
        vu, vp, vpi = v[:nU], v[nU:nU + nP], v[nU + nP:]
        zu = self.solve_uu(vu)
        zp = (vp - self.B.Aup.T @ zu) / self.Bt
        zpi = self.solve_pi(vpi - self.B.dt * (self.B.Appi.T @ zp))
        return np.concatenate([zu, zp, zpi])

    def matrix(self):
        """M itself (for the spectral pins)."""
        B = self.B
        return sp.bmat([[B.Auu, B.Aup, None],
                        [None, sp.diags(self.Bt), B.dt * B.Appi],
                        [None, None, self.C]], format="csr")


def build(B: Blocks, kind="amg", coarse_max=COARSE_MAX) -> Preconditioner:
    Bt = btilde(B)
    C = ctilde(B, Bt)
    pc = Preconditioner(B, Bt, C, kind)
    if kind == "exact":
        pc._luu = spla.splu(B.Auu.tocsc())
        pc._lpi = spla.splu(C.tocsc())
    elif kind == "amg_rbm":
        from . import rbm
        pc.u_levels = rbm.build_u_hierarchy(B, coarse_max)
        pc.pi_levels = build_pi_hierarchy(B, C, coarse_max)
    else:
        pc.u_levels = build_u_hierarchy(B, coarse_max)
        pc.pi_levels = build_pi_hierarchy(B, C, coarse_max)
    return pc
