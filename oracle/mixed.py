"""The mixed (non-hybridized) formulation and the block-triangular
preconditioner (BTP) that Section 5 compares against (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* Eq. (mfeSys) with the stabilization of Eq. (stab_A): unknowns u (Q1
  nodes), p (cells) and q, one continuous RT0 flux per face, oriented along
  the face's +axis.  A_qq = (phi_i, mu kappa^-1 phi_j) is assembled from the
  cell mass matrices A_ww,T of the unit-outward-flux basis with the sign of
  each local face relative to the face's axis (- on the cell's lower face,
  + on its upper face); A_qp = -(div phi_i, chi_j) = -s_lf; A_pq = -A_qp^T;
  the (p, p) block is A_pp + A_stab with A_pp = S_eps |T|.
* Unknown order [u | p | q], so that f_u and f_p are those of the hybrid
  system and f_q = 0 (homogeneous pressure data).  Reading: every face is
  kept (Table tab:grids counts n_q = all faces); on a no-flow face q = 0 is
  imposed by zeroing its row and column and keeping the diagonal, as the
  hybrid system does for prescribed interface pressures.
* BTP, Eq. (prec): M = [[M_uu, 0, 0], [0, M_qq, 0], [A_pu, dt A_pq, M_Cp]]
  (in the paper's (u, q, p) order), applied by forward substitution.
  C~_p = A_stab + A_pp + diag(A_up^T diag(A_uu)^-1 A_up) (the fixed-stress
  diagonal) - dt A_pq L_qq^-1 A_qp (= + dt A_qp^T L_qq^-1 A_qp), with L_qq
  the lumped A_qq: the Schur complement C_p of the paper with A_uu and A_qq
  replaced by diagonal approximations.  Reading of
  "lumped spectrally equivalent matrix": L_qq = diag(sum_g |A_qq[f, g]|).
* M_I^(m): exact inner solves with A_uu, A_qq and C~_p.  M_II^(m): the
  displacement V-cycle of M_II^(h); for A_qq, whose incomplete Cholesky the
  paper uses, this library's reading is Chebyshev(2) preconditioned by
  diag(A_qq) on [lmax/10, lmax] (A_qq is spectrally equivalent to its
  diagonal, and a polynomial needs no triangular solves); for C~_p, the
  scalar smoothed-aggregation multigrid of the cell levels of M_II^(h)'s
  interface-pressure hierarchy, started at C~_p on the cell lattice.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import precond
from .system import Blocks, _dirichlet

FACE_SIGN = np.array([-1.0, 1.0, -1.0, 1.0, -1.0, 1.0])


@dataclass
class Mixed:
    B: Blocks
    Aqq: sp.csr_matrix
    Aqp: sp.csr_matrix
    Apq: sp.csr_matrix
    q_fixed: np.ndarray            # bool per face: no-flow (q = 0)

    @property
    def sizes(self):
        nU, nP, nF = self.B.sizes
        return nU, nP, nF


def assemble_mixed(B: Blocks, face_bc) -> Mixed:
    mesh = B.mesh
    nT, nF = mesh.n_cells, mesh.n_faces
    cf = mesh.cell_faces
    s = np.tile(FACE_SIGN, (nT, 1))
    R = np.repeat(cf, 6, axis=1).ravel()
    C = np.tile(cf, (1, 6)).ravel()
    V = (s[:, :, None] * B.Aww_cells * s[:, None, :]).ravel()
    Aqq = sp.csr_matrix((V, (R, C)), shape=(nF, nF))
    Aqq.sum_duplicates()
    Aqp = sp.csr_matrix((-s.ravel(), (cf.ravel(), np.repeat(np.arange(nT), 6))), shape=(nF, nT))
    q_fixed = (np.asarray(face_bc) & 4) != 0
    dq = Aqq.diagonal()
    Aqq = _dirichlet(Aqq, q_fixed, q_fixed, np.where(q_fixed, dq, 0.0))
    Aqp = _dirichlet(Aqp, q_fixed, None, None)
    Apq = (-Aqp.T).tocsr()
    return Mixed(B, Aqq, Aqp, Apq, q_fixed)


def mixed_matrix(M: Mixed) -> sp.csr_matrix:
    """Eq. (mfeSys) + stabilization, unknowns [u | p | q]."""
    B = M.B
    return sp.bmat([[B.Auu, B.Aup, None],
                    [B.Apu, B.App + B.Astab, B.dt * M.Apq],
                    [None, M.Aqp, M.Aqq]], format="csr")


def solve_direct(M: Mixed, b):
    """x = A_M^-1 b (LU of the |diag|^-1/2-scaled matrix, two refinement
    steps, as oracle.solve_direct)."""
    A = mixed_matrix(M).tocsc()
    d = 1.0 / np.sqrt(np.abs(A.diagonal()))
    D = sp.diags(d)
    lu = spla.splu((D @ A @ D).tocsc())
    x = d * lu.solve(d * b)
    for _ in range(2):
        x = x + d * lu.solve(d * (b - A @ x))
    return x


def lumped_qq(M: Mixed) -> np.ndarray:
    return np.asarray(abs(M.Aqq).sum(axis=1)).ravel()


def ctilde_p(M: Mixed) -> sp.csr_matrix:
    B = M.B
    dAuu = B.Auu.diagonal()
    fixed_stress = np.asarray((B.Aup.multiply(B.Aup)).T @ (1.0 / dAuu)).ravel()
    C = B.App + B.Astab + sp.diags(fixed_stress) - B.dt * (M.Apq @ sp.diags(1.0 / lumped_qq(M)) @ M.Aqp)
    C = C.tocsr()
    C.sum_duplicates()
    return C


def equilibration(M: Mixed, Cp: sp.csr_matrix) -> np.ndarray:
    """D_s = diag(A_uu, C~_p, A_qq)^(-1/2) (the stopping test's scaling)."""
    d = np.concatenate([M.B.Auu.diagonal(), Cp.diagonal(), M.Aqq.diagonal()])
    return 1.0 / np.sqrt(d)


def _cell_hierarchy(Cp: sp.csr_matrix, dims, coarse_max):
    """Smoothed-aggregation hierarchy of C~_p on the cell lattice (the
    interface-pressure spec below its face level)."""
    lev = precond.Level(Cp.tocsr(), 1, dims, active=np.ones(Cp.shape[0], bool))
    levels = [lev]
    while lev.dims[0] * lev.dims[1] * lev.dims[2] > coarse_max:
        precond._finish_level(lev)
        P, cdims, act = precond._sa_prolongator(lev)
        lev.P = P
        lev = precond.Level(precond._galerkin(P, lev.A, act), 1, cdims, active=act)
        levels.append(lev)
    precond._dense_coarse(lev)
    return levels


@dataclass
class BTP:
    M: Mixed
    Cp: sp.csr_matrix
    kind: str                      # "exact" (M_I^(m)) or "amg" (M_II^(m))
    u_levels: list = field(default_factory=list)
    q_level: precond.Level | None = None
    p_levels: list = field(default_factory=list)
    _lu: tuple = ()

    def solve_uu(self, r):
        return self._lu[0].solve(r) if self.kind == "exact" else precond.vcycle(self.u_levels, r)

    def solve_qq(self, r):
        if self.kind == "exact":
            return self._lu[1].solve(r)
        return precond.chebyshev(self.q_level, r, np.zeros_like(r))

    def solve_cp(self, r):
        return self._lu[2].solve(r) if self.kind == "exact" else precond.vcycle(self.p_levels, r)

    def apply(self, v):
        """Forward substitution with M (Eq. prec): u and q, then p."""
        nU, nP, nF = self.M.sizes
        B = self.M.B
        vu, vp, vq = v[:nU], v[nU:nU + nP], v[nU + nP:]
        zu = self.solve_uu(vu)
        zq = self.solve_qq(vq)
        zp = self.solve_cp(vp - B.Apu @ zu - B.dt * (self.M.Apq @ zq))
        return np.concatenate([zu, zp, zq])

    def matrix(self):
        """M itself, in the [u | p | q] order (for the spectral pins)."""
        B, M = self.M.B, self.M
        return sp.bmat([[B.Auu, None, None],
                        [B.Apu, self.Cp, B.dt * M.Apq],
                        [None, None, M.Aqq]], format="csr")


def build_btp(M: Mixed, kind="amg", coarse_max=precond.COARSE_MAX, Cp=None) -> BTP:
    Cp = ctilde_p(M) if Cp is None else Cp
    pc = BTP(M, Cp, kind)
    if kind == "exact":
        pc._lu = (spla.splu(M.B.Auu.tocsc()), spla.splu(M.Aqq.tocsc()), spla.splu(Cp.tocsc()))
        return pc
    mesh = M.B.mesh
    pc.u_levels = precond.build_u_hierarchy(M.B, coarse_max)
    q = precond.Level(M.Aqq.tocsr(), 1, None, active=~M.q_fixed)
    precond._finish_level(q)
    pc.q_level = q
    pc.p_levels = _cell_hierarchy(Cp, (mesh.nx, mesh.ny, mesh.nz), coarse_max)
    return pc
