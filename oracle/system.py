"""Global stabilized, condensed MHFE system and its pieces (oracle, FP64).

* Eq. (hybridSys) / Section 2.2: broken RT0 fluxes w with A_ww block
  diagonal (one SPD 6x6 block per cell), A_wp = -1, A_wpi = I in the
  unit-outward-flux basis, A_pw = -A_wp^T, A_piw = -A_wpi^T.
* Eq. (hmfeSys), Eq. (A_33H): static condensation onto (u, p, pi):
  Abar_pp = A_pp - dt A_pw A_ww^-1 A_wp, dt A_ppi = -dt A_pw A_ww^-1 A_wpi,
  A_pip = -A_piw A_ww^-1 A_wp, A_pipi = -A_piw A_ww^-1 A_wpi.
* Eq. (J_def), Eq. (stab_A): pressure-jump stabilization on the internal
  faces of each macro-element, beta_M = (3b)^2 / [32 (lambda + 4G)].
* Section 2.1: backward Euler, f~_n = b div u_{n-1} + S_eps p_{n-1}.
* Appendix A: right-hand sides (tractions, prescribed fluxes).

Readings where the paper is silent: all dofs are kept and homogeneous
Dirichlet data is imposed by zeroing the row and column and keeping the
diagonal; Lame parameters and b of a macro-element are cell-volume averages;
the stabilization acts on p_n only (no A_stab p_{n-1} term).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import elements as el
from .mesh import LOCAL_FACE_NODES, Mesh


@dataclass
class Blocks:
    mesh: Mesh
    dt: float
    Auu: sp.csr_matrix
    Aup: sp.csr_matrix
    Apu: sp.csr_matrix
    App: sp.csr_matrix         # S_eps |T| (diagonal)
    Abar_pp: sp.csr_matrix     # A_pp - dt A_pw A_ww^-1 A_wp (diagonal)
    Astab: sp.csr_matrix
    Appi: sp.csr_matrix        # dt A_ppi is the (p, pi) block
    Apip: sp.csr_matrix
    Apipi: sp.csr_matrix
    Aww_cells: np.ndarray      # (n_T, 6, 6)
    Dw: np.ndarray             # diag(A_wp^T A_ww^-1 A_wp) per cell = 1^T W 1
    vol: np.ndarray
    u_fixed: np.ndarray        # bool (n_u,)
    pi_fixed: np.ndarray       # bool (n_pi,)
    f_u: np.ndarray            # traction load (constant in time)
    beta: np.ndarray           # beta_M per macro
    macro_vol: np.ndarray

    @property
    def sizes(self):
        return self.Auu.shape[0], self.App.shape[0], self.Apipi.shape[0]


def _dirichlet(A, rows_fixed, cols_fixed, keep_diag):
    A = A.tocsr().copy()
    if rows_fixed is not None:
        r = sp.diags((~rows_fixed).astype(float))
        A = (r @ A)
    if cols_fixed is not None:
        c = sp.diags((~cols_fixed).astype(float))
        A = (A @ c)
    if keep_diag is not None:
        d = keep_diag
        A = A + sp.diags(d)
    A = A.tocsr()
    A.eliminate_zeros()
    return A


def assemble(prob) -> Blocks:
    mesh = Mesh(prob.nx, prob.ny, prob.nz, prob.coords)
    nT, nF, nN = mesh.n_cells, mesh.n_faces, mesh.n_nodes
    nU = 3 * nN
    X = mesh.element_coords()

    Ke, Aup_e, vol, detmin = el.q1_element(X, prob.E, prob.nu, prob.biot)
    if np.any(detmin <= 0):
        raise ValueError("inverted or degenerate element")
    dofs = (3 * mesh.cell_nodes[:, :, None] + np.arange(3)[None, None, :]).reshape(nT, 24)
    rows = np.repeat(dofs, 24, axis=1).ravel()
    cols = np.tile(dofs, (1, 24)).ravel()
    Auu = sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(nU, nU))
    Aup = sp.csr_matrix((Aup_e.ravel(), (dofs.ravel(), np.repeat(np.arange(nT), 24))), shape=(nU, nT))

    # RT0 condensation, cell by cell
    Aww = el.rt0_element(X, prob.mu, prob.kappa)
    W = np.linalg.inv(Aww)
    one = np.ones(6)
    W1 = W @ one                               # (n,6)
    Dw = W1 @ one                              # 1^T W 1
    App = sp.diags(prob.Seps * vol).tocsr()
    Abar = sp.diags(prob.Seps * vol + prob.dt * Dw).tocsr()
    cf = mesh.cell_faces
    Appi = sp.csr_matrix(((-W1).ravel(), (np.repeat(np.arange(nT), 6), cf.ravel())), shape=(nT, nF))
    Apip = sp.csr_matrix(((-W1).ravel(), (cf.ravel(), np.repeat(np.arange(nT), 6))), shape=(nF, nT))
    Apipi = sp.csr_matrix((W.ravel(), (np.repeat(cf, 6, axis=1).ravel(), np.tile(cf, (1, 6)).ravel())),
                          shape=(nF, nF))

    # macro-element stabilization
    lam, G = el.lame(prob.E, prob.nu)
    nM = mesh.n_macros
    mvol = np.bincount(mesh.cell_macro, weights=vol, minlength=nM)
    lam_M = np.bincount(mesh.cell_macro, weights=lam * vol, minlength=nM) / mvol
    G_M = np.bincount(mesh.cell_macro, weights=G * vol, minlength=nM) / mvol
    b_M = np.bincount(mesh.cell_macro, weights=prob.biot * vol, minlength=nM) / mvol
    beta = (3.0 * b_M) ** 2 / (32.0 * (lam_M + 4.0 * G_M))
    k, l, m = mesh.internal_macro_faces()
    c = beta[m] * mvol[m]
    Astab = sp.csr_matrix((np.concatenate([c, c, -c, -c]),
                           (np.concatenate([k, l, k, l]), np.concatenate([k, l, l, k]))), shape=(nT, nT))

    # boundary conditions
    u_fixed = np.zeros(nU, bool)
    for comp in range(3):
        u_fixed[3 * np.arange(nN) + comp] = (prob.node_fix >> comp) & 1 == 1
    pi_fixed = (prob.face_bc & 2) != 0

    Auu_d = Auu.diagonal()
    Auu = _dirichlet(Auu, u_fixed, u_fixed, np.where(u_fixed, Auu_d, 0.0))
    Aup = _dirichlet(Aup, u_fixed, None, None)
    Apu = (-Aup.T).tocsr()
    Apipi_d = Apipi.diagonal()
    Apipi = _dirichlet(Apipi, pi_fixed, pi_fixed, np.where(pi_fixed, Apipi_d, 0.0))
    Appi = _dirichlet(Appi, None, pi_fixed, None)
    Apip = _dirichlet(Apip, pi_fixed, None, None)

    # traction load f_u = (eta_i, t)_Gamma_sigma
    f_u = np.zeros(nU)
    trac = np.flatnonzero(prob.face_bc & 1)
    for f in trac:
        slot = 0 if mesh.face_cells[f, 0] >= 0 else 1
        cell, lf = mesh.face_cells[f, slot], mesh.face_local[f, slot]
        loc = LOCAL_FACE_NODES[lf]   # ordered by the two in-face offsets
        Xf = X[cell, loc][None]
        contrib = el.face_load(Xf, prob.traction)[0]
        for a, ln in enumerate(loc):
            n = mesh.cell_nodes[cell, ln]
            f_u[3 * n:3 * n + 3] += contrib[a]
    f_u[u_fixed] = 0.0

    return Blocks(mesh, prob.dt, Auu, Aup, Apu, App, Abar, Astab, Appi, Apip, Apipi,
                  Aww, Dw, vol, u_fixed, pi_fixed, f_u, beta, mvol)


def system_matrix(B: Blocks) -> sp.csr_matrix:
    """Eq. (stab_A), hybrid form: [[A_uu, A_up, 0], [A_pu, Abar_pp + A_stab,
    dt A_ppi], [0, A_pip, A_pipi]]."""
    return sp.bmat([[B.Auu, B.Aup, None],
                    [B.Apu, B.Abar_pp + B.Astab, B.dt * B.Appi],
                    [None, B.Apip, B.Apipi]], format="csr")


def rhs(B: Blocks, u_prev=None, p_prev=None, load_scale=1.0) -> np.ndarray:
    """Eq. (hmfeSys) right-hand side with f_w = 0 (homogeneous pressure data)
    and f_pi = 0 (no-flow): [f_u ; A_pu u_{n-1} + S_eps |T| p_{n-1} ; 0]."""
    nU, nP, nPi = B.sizes
    fp = np.zeros(nP)
    if u_prev is not None:
        fp += B.Apu @ u_prev
    if p_prev is not None:
        fp += B.App @ p_prev
    return np.concatenate([load_scale * B.f_u, fp, np.zeros(nPi)])


def split(B: Blocks, x):
    nU, nP, nPi = B.sizes
    return x[:nU], x[nU:nU + nP], x[nU + nP:]


def reconstruct_fluxes(B: Blocks, p, pi) -> np.ndarray:
    """Section 2.2: cell-based recovery w_T = A_ww,T^-1 (-A_wp p - A_wpi pi)
    = W_T (p_T 1 - pi_T) (outward fluxes, zero prescribed pressure)."""
    W = np.linalg.inv(B.Aww_cells)
    pi_T = pi[B.mesh.cell_faces]
    return np.einsum("nij,nj->ni", W, p[:, None] - pi_T)


def hybrid_uncondensed(prob, B: Blocks) -> tuple[sp.csr_matrix, int]:
    """Eq. (hybridSys) before condensation, unknowns (u, w, p, pi), with the
    same Dirichlet treatment; used to pin the static condensation."""
    mesh = B.mesh
    nU, nP, nPi = B.sizes
    nW = 6 * nP
    Aww = sp.block_diag(list(B.Aww_cells), format="csr")
    Awp = sp.csr_matrix((-np.ones(nW), (np.arange(nW), np.repeat(np.arange(nP), 6))), shape=(nW, nP))
    Awpi = sp.csr_matrix((np.ones(nW), (np.arange(nW), mesh.cell_faces.ravel())), shape=(nW, nPi))
    Awpi = _dirichlet(Awpi, None, B.pi_fixed, None)
    Apw = (-Awp.T).tocsr()
    Apiw = (-Awpi.T).tocsr()
    # Dirichlet faces: identity-like row keeps the system square and nonsingular
    Dfix = sp.diags(np.where(B.pi_fixed, 1.0, 0.0))
    A = sp.bmat([[B.Auu, None, B.Aup, None],
                 [None, Aww, Awp, Awpi],
                 [B.Apu, B.dt * Apw, B.App + B.Astab, None],
                 [None, Apiw, None, Dfix]], format="csr")
    return A, nW
