"""Structured hexahedral mesh topology for the oracle (test infrastructure).

Section 2: the partition T_h into n_T hexahedra, the face set E_h, one
P0 pressure per cell, one Lagrange multiplier per face, Q1 nodes.
Section 3 / Fig. 1: macro-elements are 2x2x2 patches of cells; this oracle
reads trailing partial patches (odd n) as macro-elements of their own.
"""
from __future__ import annotations

import numpy as np

# local node a = di + 2*dj + 4*dk, reference coordinate (2di-1, 2dj-1, 2dk-1)
LOCAL_NODE_OFFSETS = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)])
# local faces: 0 x-, 1 x+, 2 y-, 3 y+, 4 z-, 5 z+
LOCAL_FACE_NODES = [
    [a for a in range(8) if LOCAL_NODE_OFFSETS[a, 0] == 0],
    [a for a in range(8) if LOCAL_NODE_OFFSETS[a, 0] == 1],
    [a for a in range(8) if LOCAL_NODE_OFFSETS[a, 1] == 0],
    [a for a in range(8) if LOCAL_NODE_OFFSETS[a, 1] == 1],
    [a for a in range(8) if LOCAL_NODE_OFFSETS[a, 2] == 0],
    [a for a in range(8) if LOCAL_NODE_OFFSETS[a, 2] == 1],
]


class Mesh:
    def __init__(self, nx: int, ny: int, nz: int, coords: np.ndarray):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.coords = np.asarray(coords, dtype=np.float64)
        self.n_nodes = (nx + 1) * (ny + 1) * (nz + 1)
        self.n_cells = nx * ny * nz
        self.nfx = (nx + 1) * ny * nz
        self.nfy = nx * (ny + 1) * nz
        self.nfz = nx * ny * (nz + 1)
        self.n_faces = self.nfx + self.nfy + self.nfz
        assert self.coords.shape == (self.n_nodes, 3)

        c = np.arange(self.n_cells)
        self.ci = c % nx
        self.cj = (c // nx) % ny
        self.ck = c // (nx * ny)
        i, j, k = self.ci, self.cj, self.ck

        def node(ii, jj, kk):
            return ii + (nx + 1) * (jj + (ny + 1) * kk)

        self.cell_nodes = np.stack(
            [node(i + o[0], j + o[1], k + o[2]) for o in LOCAL_NODE_OFFSETS], axis=1)

        fx = lambda ii, jj, kk: ii + (nx + 1) * (jj + ny * kk)
        fy = lambda ii, jj, kk: self.nfx + ii + nx * (jj + (ny + 1) * kk)
        fz = lambda ii, jj, kk: self.nfx + self.nfy + ii + nx * (jj + ny * kk)
        self.cell_faces = np.stack(
            [fx(i, j, k), fx(i + 1, j, k), fy(i, j, k), fy(i, j + 1, k), fz(i, j, k), fz(i, j, k + 1)],
            axis=1)

        # face -> (cell, local face) pairs; -1 where the face is on the boundary
        self.face_cells = -np.ones((self.n_faces, 2), dtype=np.int64)
        self.face_local = -np.ones((self.n_faces, 2), dtype=np.int64)
        for lf in range(6):
            f = self.cell_faces[:, lf]
            slot = 1 if lf % 2 == 0 else 0  # the cell on the face's + side is slot 1
            self.face_cells[f, slot] = c
            self.face_local[f, slot] = lf

        # macro-element index (i>>1, j>>1, k>>1)
        mx, my = (nx + 1) // 2, (ny + 1) // 2
        self.n_macros = mx * my * ((nz + 1) // 2)
        self.cell_macro = (i >> 1) + mx * ((j >> 1) + my * (k >> 1))

    def element_coords(self) -> np.ndarray:
        """(n_T, 8, 3) node coordinates per cell in local order."""
        return self.coords[self.cell_nodes]

    def internal_macro_faces(self):
        """Faces e in Gamma_M (between two cells of one macro-element):
        returns arrays (cell_k, cell_l, macro)."""
        fc = self.face_cells
        both = (fc[:, 0] >= 0) & (fc[:, 1] >= 0)
        k, l = fc[both, 0], fc[both, 1]
        same = self.cell_macro[k] == self.cell_macro[l]
        return k[same], l[same], self.cell_macro[k[same]]
