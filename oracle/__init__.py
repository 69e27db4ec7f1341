"""FP64 CPU oracle for the stabilized, hybridized Q1-RT0-P0 poromechanics
solve of Frigo, Castelletto, Ferronato & White (arXiv:2002.09603).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
or run anything in this package.  The CUDA library shares no code with it:
the two meet only through the seeded inputs of ``mhfp_inputs``.

Plain numpy / scipy in FP64, written from the paper:

* ``mesh``     structured hexahedral topology, macro-elements (Section 3)
* ``elements`` Q1 stiffness and coupling, RT0 mass (Appendix A)
* ``system``   static condensation (Eq. hmfeSys, A_33H), stabilization
               (Eq. J_def, stab_A), boundary conditions, right-hand side,
               flux reconstruction, the uncondensed hybrid system
* ``precond``  B~_p, C~_pi, the block-triangular preconditioner (Eq.
               hybridPrec) with exact inner solves (M_I^(h)) or with this
               library's multigrid spec (parity unpinned by the paper)
* ``rbm``      the M_III^(h) displacement multigrid: smoothed aggregation
               with the six rigid-body modes as near-kernel (Section 5;
               parity unpinned by the paper)
* ``fgmres``   right-preconditioned flexible GMRES (Section 5)
"""
from . import elements, fgmres, mesh, precond, system  # noqa: F401
from .system import assemble, rhs, system_matrix  # noqa: F401


def solve_direct(B, b, refine=2):
    """The plain definition of the per-step result: x = A_H^-1 b.

    The blocks of A_H differ by many orders of magnitude (stiffness vs.
    kappa h / mu), so the LU is taken of the symmetrically scaled matrix
    D A_H D with D = |diag(A_H)|^(-1/2), followed by `refine` steps of
    iterative refinement on the unscaled residual."""
    import numpy as np
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    A = system_matrix(B).tocsc()
    d = 1.0 / np.sqrt(np.abs(A.diagonal()))
    D = sp.diags(d)
    lu = spla.splu((D @ A @ D).tocsc())
    x = d * lu.solve(d * b)
    for _ in range(refine):
        x = x + d * lu.solve(d * (b - A @ x))
    return x


def time_steps(prob, nsteps, kind="direct", tol=1e-10, restart=50, load_scale=1.0):
    """Backward-Euler steps n = 1..nsteps from u_0 = 0, p_0 = 0 (Section 2.1).
    Returns the list of solution vectors and per-step solver info."""
    import numpy as np
    B = assemble(prob)
    nU, nP, nPi = B.sizes
    xs, infos = [], []
    u_prev, p_prev = np.zeros(nU), np.zeros(nP)
    A = system_matrix(B)
    pc = None if kind == "direct" else precond.build(B, kind)
    for _ in range(nsteps):
        b = rhs(B, u_prev, p_prev, load_scale)
        if pc is None:
            x = solve_direct(B, b)
            info = {}
        else:
            s = precond.equilibration(B, pc.Bt, pc.C)
            x, info = fgmres.fgmres(lambda v: A @ v, pc.apply, b, tol=tol, restart=restart, scale=s)
        xs.append(x)
        infos.append(info)
        u_prev, p_prev = x[:nU], x[nU:nU + nP]
    return xs, infos
