"""Seeded synthetic inputs for the hybridized poromechanics solve.

This module only *describes* problems: structured hexahedral meshes of a box,
boundary-condition masks, per-cell material fields and the time-step size.
It holds none of the method's arithmetic (no element integrals, no assembly,
no solver) and is the one piece shared by the FP64 oracle, the CUDA path,
the tests and the benchmark, so that both sides see bit-identical inputs.

Numbering (shared convention, the paper leaves it open):

* nodes  ``n = i + (nx+1)*(j + (ny+1)*k)``, ``0<=i<=nx`` ...
* cells  ``c = i + nx*(j + ny*k)``
* faces  x-normal family first, then y-normal, then z-normal, each
  lexicographic in its own index box (x family: ``0<=i<=nx, j<ny, k<nz``).

Boundary masks:

* ``node_fix[n]`` bit0/bit1/bit2 = ux/uy/uz prescribed to zero (rollers,
  clamps).  Only homogeneous displacement data is supported.
* ``face_bc[f]`` bit0 = traction face (the uniform traction vector
  ``traction`` acts on it), bit1 = drained face (interface pressure prescribed
  to zero), bit2 = explicit no-flow face.  Interior faces are 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

FIX_X, FIX_Y, FIX_Z = 1, 2, 4
BC_TRACTION, BC_DRAINED, BC_NOFLOW = 1, 2, 4


@dataclass
class Problem:
    nx: int
    ny: int
    nz: int
    coords: np.ndarray          # (n_nodes, 3) float64
    node_fix: np.ndarray        # (n_nodes,) uint8
    face_bc: np.ndarray         # (n_faces,) uint8
    E: np.ndarray               # (n_cells,) Young modulus [Pa]
    nu: np.ndarray              # (n_cells,) Poisson ratio
    biot: np.ndarray            # (n_cells,) Biot coefficient
    Seps: np.ndarray            # (n_cells,) constrained specific storage [1/Pa]
    mu: np.ndarray              # (n_cells,) fluid viscosity [Pa s]
    kappa: np.ndarray           # (n_cells, 3) diagonal permeability [m^2]
    dt: float
    traction: np.ndarray = field(default_factory=lambda: np.array([0.0, 0.0, -1.0]))
    name: str = ""

    @property
    def n_nodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_faces(self) -> int:
        nx, ny, nz = self.nx, self.ny, self.nz
        return (nx + 1) * ny * nz + nx * (ny + 1) * nz + nx * ny * (nz + 1)

    @property
    def sizes(self) -> tuple[int, int, int]:
        """(n_u, n_p, n_pi): all dofs are kept, Dirichlet ones included."""
        return 3 * self.n_nodes, self.n_cells, self.n_faces


def _face_offsets(nx, ny, nz):
    nfx = (nx + 1) * ny * nz
    nfy = nx * (ny + 1) * nz
    return nfx, nfy


def boundary_face_ids(nx, ny, nz, side: str) -> np.ndarray:
    """Indices of the boundary faces on one side of the box ('x0','x1',...,'z1')."""
    nfx, nfy = _face_offsets(nx, ny, nz)
    axis, end = side[0], side[1] == "1"
    if axis == "x":
        i = nx if end else 0
        j, k = np.meshgrid(np.arange(ny), np.arange(nz), indexing="ij")
        return (i + (nx + 1) * (j + ny * k)).ravel()
    if axis == "y":
        j = ny if end else 0
        i, k = np.meshgrid(np.arange(nx), np.arange(nz), indexing="ij")
        return (nfx + i + nx * (j + (ny + 1) * k)).ravel()
    k = nz if end else 0
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    return (nfx + nfy + i + nx * (j + ny * k)).ravel()


def boundary_node_ids(nx, ny, nz, side: str) -> np.ndarray:
    idx = np.arange((nx + 1) * (ny + 1) * (nz + 1))
    i = idx % (nx + 1)
    j = (idx // (nx + 1)) % (ny + 1)
    k = idx // ((nx + 1) * (ny + 1))
    axis, end = side[0], side[1] == "1"
    v = {"x": (i, nx), "y": (j, ny), "z": (k, nz)}[axis]
    return idx[v[0] == (v[1] if end else 0)]


def box_coords(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0) -> np.ndarray:
    x = np.linspace(0.0, lx, nx + 1)
    y = np.linspace(0.0, ly, ny + 1)
    z = np.linspace(0.0, lz, nz + 1)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).copy()


def jitter_coords(coords, nx, ny, nz, amp, rng) -> np.ndarray:
    """Move every node by U(-amp*h, amp*h) per coordinate, except along the
    normal of any boundary plane it lies on (so rollers stay planar)."""
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    d = rng.uniform(-amp, amp, size=coords.shape) * h
    idx = np.arange(coords.shape[0])
    ijk = [idx % (nx + 1), (idx // (nx + 1)) % (ny + 1), idx // ((nx + 1) * (ny + 1))]
    for a, n in enumerate((nx, ny, nz)):
        on = (ijk[a] == 0) | (ijk[a] == n)
        d[on, a] = 0.0
    return coords + d


def gaussian_field_exp(n, sigma, ell, rng) -> np.ndarray:
    """Stationary Gaussian field on an n^3 cell grid with covariance
    sigma^2 exp(-r/ell) (r in cell units), by circulant embedding on a
    (2n)^3 periodic grid.  Returns (n^3,) in cell order (i fastest)."""
    m = 2 * n
    g = np.arange(m)
    g = np.minimum(g, m - g).astype(np.float64)
    r = np.sqrt(g[:, None, None] ** 2 + g[None, :, None] ** 2 + g[None, None, :] ** 2)
    cov = sigma * sigma * np.exp(-r / ell)
    lam = np.fft.fftn(cov).real
    lam = np.maximum(lam, 0.0)
    xi = rng.standard_normal((m, m, m)) + 1j * rng.standard_normal((m, m, m))
    f = np.fft.ifftn(np.sqrt(lam) * xi) * np.sqrt(m ** 3)
    f = f.real[:n, :n, :n]  # axes (k, j, i)
    return np.ascontiguousarray(f).ravel()


def _materials(nT, E, nu, b, S, mu, kappa):
    full = lambda v: np.full(nT, float(v))
    k = np.asarray(kappa, dtype=np.float64)
    if k.ndim == 0:
        k = np.full((nT, 3), float(k))
    elif k.ndim == 1:
        k = np.repeat(k[:, None], 3, axis=1)
    return dict(E=full(E) if np.ndim(E) == 0 else np.asarray(E, float),
                nu=full(nu) if np.ndim(nu) == 0 else np.asarray(nu, float),
                biot=full(b), Seps=full(S) if np.ndim(S) == 0 else np.asarray(S, float),
                mu=full(mu), kappa=np.ascontiguousarray(k))


def terzaghi_bcs(nx, ny, nz):
    """Rollers on x=0,1 / y=0,1 / z=0, loaded and drained top z=1, no-flow
    elsewhere (a consolidation column)."""
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    fix = np.zeros(nn, np.uint8)
    for s, bit in (("x0", FIX_X), ("x1", FIX_X), ("y0", FIX_Y), ("y1", FIX_Y), ("z0", FIX_Z)):
        fix[boundary_node_ids(nx, ny, nz, s)] |= bit
    nfx, nfy = _face_offsets(nx, ny, nz)
    nf = nfx + nfy + nx * ny * (nz + 1)
    fbc = np.zeros(nf, np.uint8)
    for s in ("x0", "x1", "y0", "y1", "z0"):
        fbc[boundary_face_ids(nx, ny, nz, s)] |= BC_NOFLOW
    fbc[boundary_face_ids(nx, ny, nz, "z1")] |= BC_TRACTION | BC_DRAINED
    return fix, fbc


def cantilever_bcs(nx, ny, nz):
    """Clamped x=0 face, loaded top z=1, no-flow on every boundary face."""
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    fix = np.zeros(nn, np.uint8)
    fix[boundary_node_ids(nx, ny, nz, "x0")] |= FIX_X | FIX_Y | FIX_Z
    nfx, nfy = _face_offsets(nx, ny, nz)
    nf = nfx + nfy + nx * ny * (nz + 1)
    fbc = np.zeros(nf, np.uint8)
    for s in ("x0", "x1", "y0", "y1", "z0", "z1"):
        fbc[boundary_face_ids(nx, ny, nz, s)] |= BC_NOFLOW
    fbc[boundary_face_ids(nx, ny, nz, "z1")] |= BC_TRACTION
    return fix, fbc


def terzaghi_cube(n=8, E=1e4, nu=0.25, b=1.0, S=1e-4, mu=1e-3, kappa=1e-12,
                  dt=1.0, load=1.0, nx=None, ny=None, nz=None) -> Problem:
    """Unit cube (or box nx*ny*nz) consolidation column, homogeneous materials.
    Defaults: the 8x8x8 plain-FP64 workload (one step of dt = 1 s)."""
    nx = n if nx is None else nx
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    fix, fbc = terzaghi_bcs(nx, ny, nz)
    mats = _materials(nx * ny * nz, E, nu, b, S, mu, kappa)
    return Problem(nx, ny, nz, box_coords(nx, ny, nz), fix, fbc, dt=float(dt),
                   traction=np.array([0.0, 0.0, -float(load)]), name=f"terzaghi-{nx}x{ny}x{nz}", **mats)


def lognormal_cube(n=64, seed=2, sigma=2.0, ell=8.0, kappa_mean=1e-13, S=0.0,
                   dt=1e-3, E=1e4, nu=0.25, b=1.0, mu=1e-3, load=1.0) -> Problem:
    """n^3 unit cube with a log-normal isotropic permeability field
    (ln kappa ~ N(ln kappa_mean, sigma^2), exponential covariance of length
    ell cells), near-undrained S_eps = 0, consolidation-column boundaries.
    Defaults: the 64^3 FP64-vs-FP32 workload."""
    rng = np.random.default_rng(seed)
    g = gaussian_field_exp(n, sigma, ell, rng)
    kap = np.exp(np.log(kappa_mean) + g)
    fix, fbc = terzaghi_bcs(n, n, n)
    mats = _materials(n ** 3, E, nu, b, S, mu, kap)
    return Problem(n, n, n, box_coords(n, n, n), fix, fbc, dt=float(dt),
                   traction=np.array([0.0, 0.0, -float(load)]), name=f"lognormal-{n}^3-s{seed}", **mats)


def layered_jitter_cube(n=128, seed=3, layers=8, jitter=0.2, dt=0.1, b=1.0, mu=1e-3,
                        load=1.0) -> Problem:
    """n^3 unit cube, interior node jitter U(+-jitter*h), `layers` horizontal
    slabs with kappa log-U[1e-18,1e-12], E log-U[1e8,1e10], nu U[0.2,0.35],
    S_eps = 0.  Defaults: the 128^3 jittered, layered workload."""
    rng = np.random.default_rng(seed)
    kl = np.exp(rng.uniform(np.log(1e-18), np.log(1e-12), layers))
    El = np.exp(rng.uniform(np.log(1e8), np.log(1e10), layers))
    nl = rng.uniform(0.2, 0.35, layers)
    coords = jitter_coords(box_coords(n, n, n), n, n, n, jitter, rng)
    k = np.arange(n ** 3) // (n * n)
    lay = (k * layers) // n
    fix, fbc = terzaghi_bcs(n, n, n)
    mats = _materials(n ** 3, El[lay], nl[lay], b, 0.0, mu, kl[lay])
    return Problem(n, n, n, coords, fix, fbc, dt=float(dt),
                   traction=np.array([0.0, 0.0, -float(load)]), name=f"layered-{n}^3-s{seed}", **mats)


def cantilever_cube(n=10, dt=0.1, E=1e5, nu=0.4, b=1.0, S=0.0, kappa=1e-7, mu=1e-3,
                    load=1.0) -> Problem:
    """3D cantilever of the paper's Test 2: unit cube clamped at x=0, loaded
    on top, no-flow everywhere."""
    fix, fbc = cantilever_bcs(n, n, n)
    mats = _materials(n ** 3, E, nu, b, S, mu, kappa)
    return Problem(n, n, n, box_coords(n, n, n), fix, fbc, dt=float(dt),
                   traction=np.array([0.0, 0.0, -float(load)]), name=f"cantilever-{n}^3", **mats)


def random_small(nx, ny, nz, seed, jitter=0.0, S=1e-4, dt=0.1) -> Problem:
    """Small heterogeneous box for parity tests: per-cell E, nu, S_eps and an
    anisotropic diagonal permeability, optional node jitter."""
    rng = np.random.default_rng(seed)
    nT = nx * ny * nz
    coords = box_coords(nx, ny, nz)
    if jitter > 0:
        coords = jitter_coords(coords, nx, ny, nz, jitter, rng)
    E = np.exp(rng.uniform(np.log(1e3), np.log(1e5), nT))
    nu = rng.uniform(0.1, 0.4, nT)
    Sv = S * np.exp(rng.uniform(-1, 1, nT))
    kap = np.exp(rng.uniform(np.log(1e-13), np.log(1e-10), (nT, 3)))
    fix, fbc = terzaghi_bcs(nx, ny, nz)
    mats = _materials(nT, E, nu, 1.0, Sv, 1e-3, kap)
    return Problem(nx, ny, nz, coords, fix, fbc, dt=float(dt),
                   traction=np.array([0.0, 0.0, -1.0]), name=f"random-{nx}x{ny}x{nz}-s{seed}", **mats)


def state_vector(rng, prob: Problem) -> np.ndarray:
    """A seeded random vector in the solver's layout [u (node-major) | p | pi]."""
    nu_, np_, npi = prob.sizes
    return rng.standard_normal(nu_ + np_ + npi)


def batch_instances(count=48, seed=4, nmin=16, nmax=64, sigma=1.5, ell=8.0, kappa_mean=1e-13, dt=1e-3):
    """`count` independent cube problems of uneven size n ~ U{nmin..nmax}
    (seeded), each with its own log-normal permeability field (sigma, ell
    cells), S_eps = 0, consolidation-column boundaries.  The batched workload
    solves each for the loads LOAD_SCALES."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(nmin, nmax + 1, size=count)
    seeds = rng.integers(0, 2 ** 31 - 1, size=count)
    return [lognormal_cube(int(n), seed=int(s), sigma=sigma, ell=ell, kappa_mean=kappa_mean, dt=dt)
            for n, s in zip(sizes, seeds)]


LOAD_SCALES = (0.5, 1.0, 2.0, 4.0)
