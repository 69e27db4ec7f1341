"""Element matrices of the Q1-RT0-P0 discretization (oracle, FP64).

Appendix A (element contributions of A_uu, A_up, A_ww, A_wp, A_wpi) and
Section 2.2 (hybridized RT0 with one flux per element face).  Quadrature is
2x2x2 Gauss-Legendre on the reference cube [-1,1]^3 (the paper does not
state one; this rule is exact on parallelepipeds).  Everything is
vectorised over cells but evaluated point by point in the textbook form.
"""
from __future__ import annotations

import numpy as np

from .mesh import LOCAL_NODE_OFFSETS

GP = 1.0 / np.sqrt(3.0)
GAUSS_POINTS = np.array([[sx * GP, sy * GP, sz * GP]
                         for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)])
GAUSS_WEIGHTS = np.ones(8)
XI_NODES = 2.0 * LOCAL_NODE_OFFSETS - 1.0  # (8,3) reference node coordinates


def q1_shape(xi):
    """Trilinear shape functions and reference gradients at one point."""
    N = np.prod(1.0 + XI_NODES * xi[None, :], axis=1) / 8.0
    dN = np.empty((8, 3))
    for d in range(3):
        others = [e for e in range(3) if e != d]
        dN[:, d] = XI_NODES[:, d] * np.prod(1.0 + XI_NODES[:, others] * xi[None, others], axis=1) / 8.0
    return N, dN


def lame(E, nu):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    G = E / (2.0 * (1.0 + nu))
    return lam, G


def _voigt_D(lam, G):
    """(n,6,6) isotropic drained elasticity C_dr in Voigt notation
    (xx, yy, zz, yz, xz, xy; engineering shear strains)."""
    n = lam.shape[0]
    D = np.zeros((n, 6, 6))
    for a in range(3):
        for b in range(3):
            D[:, a, b] = lam
        D[:, a, a] = lam + 2.0 * G
    for a in range(3, 6):
        D[:, a, a] = G
    return D


def _B_matrix(dNdx):
    """(n,8,3) physical gradients -> (n,6,24) strain-displacement matrix,
    dof ordering 3*a + component."""
    n = dNdx.shape[0]
    B = np.zeros((n, 6, 24))
    for a in range(8):
        gx, gy, gz = dNdx[:, a, 0], dNdx[:, a, 1], dNdx[:, a, 2]
        B[:, 0, 3 * a + 0] = gx
        B[:, 1, 3 * a + 1] = gy
        B[:, 2, 3 * a + 2] = gz
        B[:, 3, 3 * a + 1] = gz
        B[:, 3, 3 * a + 2] = gy
        B[:, 4, 3 * a + 0] = gz
        B[:, 4, 3 * a + 2] = gx
        B[:, 5, 3 * a + 0] = gy
        B[:, 5, 3 * a + 1] = gx
    return B


def jacobians(X, xi):
    """J_ij = d x_i / d xi_j at reference point xi for all cells; X (n,8,3)."""
    _, dN = q1_shape(xi)
    return np.einsum("nai,aj->nij", X, dN)


def q1_element(X, E, nu, biot):
    """Appendix A: [A_uu]_ab = (grad^s eta_a, C_dr : grad^s eta_b)_T and
    [A_up]_a = -(div eta_a, b)_T, plus |T|.

    X (n,8,3).  Returns Ke (n,24,24), Aup (n,24), vol (n,), detJ_min (n,).
    """
    n = X.shape[0]
    lam, G = lame(np.asarray(E, float), np.asarray(nu, float))
    D = _voigt_D(lam, G)
    Ke = np.zeros((n, 24, 24))
    Aup = np.zeros((n, 24))
    vol = np.zeros(n)
    detmin = np.full(n, np.inf)
    for q, w in zip(GAUSS_POINTS, GAUSS_WEIGHTS):
        _, dN = q1_shape(q)
        J = np.einsum("nai,aj->nij", X, dN)
        det = np.linalg.det(J)
        detmin = np.minimum(detmin, det)
        Jinv = np.linalg.inv(J)
        dNdx = np.einsum("aj,nji->nai", dN, Jinv)   # dN_a/dx_i = dN_a/dxi_j * dxi_j/dx_i
        B = _B_matrix(dNdx)
        Ke += (w * det)[:, None, None] * np.einsum("nsi,nst,ntj->nij", B, D, B)
        div = dNdx.reshape(n, 24)                     # div(N_a e_c) = dN_a/dx_c
        Aup += -(w * det * biot)[:, None] * div
        vol += w * det
    return Ke, Aup, vol, detmin


def rt0_reference_basis(xi):
    """Lowest-order Raviart-Thomas basis on [-1,1]^3 with unit outward flux
    through its own face: local faces x-, x+, y-, y+, z-, z+.  (6,3)."""
    phi = np.zeros((6, 3))
    for d in range(3):
        phi[2 * d, d] = -(1.0 - xi[d]) / 8.0
        phi[2 * d + 1, d] = (1.0 + xi[d]) / 8.0
    return phi


def rt0_element(X, mu, kappa):
    """Appendix A: [A_ww]_ij = (phi_i, mu kappa^{-1} phi_j)_T for the six
    broken RT0 fluxes of one cell, phi = J phi_hat / det J (contravariant
    Piola map).  kappa (n,3) diagonal.  Returns (n,6,6)."""
    n = X.shape[0]
    kinv = np.asarray(mu, float)[:, None] / np.asarray(kappa, float)  # (n,3) mu / kappa
    A = np.zeros((n, 6, 6))
    for q, w in zip(GAUSS_POINTS, GAUSS_WEIGHTS):
        J = jacobians(X, q)
        det = np.linalg.det(J)
        ph = rt0_reference_basis(q)                     # (6,3)
        phys = np.einsum("nij,fj->nfi", J, ph)          # J phi_hat, (n,6,3)
        A += (w / det)[:, None, None] * np.einsum("nfi,ni,ngi->nfg", phys, kinv, phys)
    return A


def face_load(Xf, traction):
    """Integral of each bilinear face shape function times a uniform traction
    over one quadrilateral face, 2x2 Gauss.  Xf (n,4,3) nodes ordered
    (s,t) = (0,0),(1,0),(0,1),(1,1).  Returns (n,4,3)."""
    n = Xf.shape[0]
    out = np.zeros((n, 4, 3))
    st = np.array([[-1, -1], [1, -1], [-1, 1], [1, 1]], dtype=float)
    for gs in (-GP, GP):
        for gt in (-GP, GP):
            N = (1 + st[:, 0] * gs) * (1 + st[:, 1] * gt) / 4.0
            dNs = st[:, 0] * (1 + st[:, 1] * gt) / 4.0
            dNt = st[:, 1] * (1 + st[:, 0] * gs) / 4.0
            xs = np.einsum("nai,a->ni", Xf, dNs)
            xt = np.einsum("nai,a->ni", Xf, dNt)
            area = np.linalg.norm(np.cross(xs, xt), axis=1)
            out += area[:, None, None] * N[None, :, None] * np.asarray(traction)[None, None, :]
    return out
