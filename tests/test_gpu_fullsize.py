"""Parity on the benchmark workload at its full size (64^3, 1,884,739
unknowns), in the launch configuration bench.py times (FP32 V-cycles inside
FP64 FGMRES(12), coarsening limit 512, graphs, autotuned schedules).

The oracle assembles the whole 64^3 system (about 1.5 min on the host) and
checks, element by element, A_H x for a seeded x, both V-cycles and M^-1 in
the schedules the set-up autotuner picks at this size (FP32 as benched, and
FP64), then the GPU solution's equilibrated residual recomputed with the
oracle's operator, and a property that holds at any size: with S_eps = 0
and a diffusion length sqrt(c_v dt) far below h, one step leaves the column
undrained below the drained top, so p = sigma / b = 1 there.

At 128^3 (14.9 M unknowns) the oracle cannot assemble the whole system in
the test's time, so it assembles windows of 8^3 cells cut out of the
workload (interior, faces, edges and corners of the box) and checks every
row whose stencil lies inside its window: the operator, the right-hand side,
the equilibration and the residual of the GPU solutions."""
import numpy as np
import pytest

import mhfp_inputs as mi
import oracle
from oracle import precond, system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_09603_gb300 import Solver, default_options
    prob = mi.lognormal_cube(64)
    B = oracle.assemble(prob)
    A = system.system_matrix(B)
    Bt = precond.btilde(B)
    C = precond.ctilde(B, Bt)
    ds = precond.equilibration(B, Bt, C)
    opt = default_options()
    opt.precision = 1
    opt.restart = 12
    opt.coarse_max = 512
    opt.reorth = 0
    s = Solver(prob)
    s.assemble_condense()
    s.setup_precond(opt)
    yield prob, B, A, ds, s
    s.close()


def test_operator_rows_full_size(full):
    prob, B, A, ds, s = full
    x = np.random.default_rng(64).standard_normal(s.n)
    y = s.apply_operator(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = A @ x
    o = 0
    for n in B.sizes:
        assert np.abs(y[o:o + n] - ref[o:o + n]).max() <= 1e-12 * np.abs(ref[o:o + n]).max()
        o += n
    assert np.allclose(s.scalings()[1].cpu().numpy(), ds, rtol=1e-12, atol=0)
    # the float-float Arnoldi operator of the bench handle, from z in FP32:
    # every row within 2^-40 of the sum of its |terms|
    z = x.astype(np.float32).astype(np.float64)
    yff = s.apply_operator_ff(torch.from_numpy(z).cuda()).cpu().numpy()
    assert np.all(np.abs(yff - A @ z) <= 2.0 ** -40 * (abs(A) @ np.abs(z)) + 1e-300)


def _bench_options(precision, restart=12):
    from paper_2002_09603_gb300 import default_options
    opt = default_options()
    opt.precision = precision
    opt.restart = restart
    opt.coarse_max = 512
    opt.reorth = 0
    return opt


def test_vcycles_and_preconditioner_full_size(full):
    """Both V-cycles and M^-1 at 64^3, element by element against the
    oracle's multigrid built with the same coarsening limit, in the launch
    schedules the autotuner picks at this size: FP32 (the benched handle,
    1e-5) and FP64 (1e-10)."""
    from paper_2002_09603_gb300 import Solver
    prob, B, A, ds, s = full
    pc = precond.build(B, "amg", coarse_max=512)
    assert [lv.A.shape[0] for lv in pc.u_levels] == [3 * 65 ** 3, 3 * 22 ** 3, 3 * 8 ** 3]
    s64 = Solver(prob)
    s64.assemble_condense()
    s64.setup_precond(_bench_options(0))
    rng = np.random.default_rng(65)
    nU, nP, nPi = B.sizes
    bu, bpi = rng.standard_normal(nU), rng.standard_normal(nPi)
    ru, rpi = precond.vcycle(pc.u_levels, bu), precond.vcycle(pc.pi_levels, bpi)
    v = rng.standard_normal(s.n)
    rz = pc.apply(v)
    for solver, tol in ((s, 1e-5), (s64, 1e-10)):
        xu = solver.vcycle(0, torch.from_numpy(bu).cuda()).cpu().numpy()
        xpi = solver.vcycle(1, torch.from_numpy(bpi).cuda()).cpu().numpy()
        assert np.abs(xu - ru).max() <= tol * np.abs(ru).max(), (tol, np.abs(xu - ru).max() / np.abs(ru).max())
        assert np.abs(xpi - rpi).max() <= tol * np.abs(rpi).max(), (tol, np.abs(xpi - rpi).max() / np.abs(rpi).max())
        z = solver.apply_precond(torch.from_numpy(v).cuda()).cpu().numpy()
        o = 0
        for n in B.sizes:
            g, r = z[o:o + n], rz[o:o + n]
            assert np.abs(g - r).max() <= tol * np.abs(r).max(), (tol, o, np.abs(g - r).max() / np.abs(r).max())
            o += n
    s64.close()


def test_bench_solve_full_size(full):
    prob, B, A, ds, s = full
    b = s.build_rhs()
    x, st = s.solve(b, tol=1e-8)
    x = x.cpu().numpy()
    bref = system.rhs(B)
    assert np.array_equal(b.cpu().numpy() != 0, bref != 0)
    rel = np.linalg.norm(ds * (bref - A @ x)) / np.linalg.norm(ds * bref)
    assert st["converged"] and rel <= 1.05e-8 and abs(rel - st["true_rel_residual"]) <= 1e-10
    nU, nP, _ = B.sizes
    p = x[nU:nU + nP].reshape(64, 64 * 64)
    assert np.allclose(p[:60], 1.0, rtol=0, atol=1e-4)
    assert 25 <= st["iterations"] <= 40


def _window(prob, org, w):
    """The sub-problem of the w^3 cells at cell offset org (even, so the
    macro-elements stay whole) of the box problem prob, with each row's
    global index and whether its stencil lies inside the window: rows of
    nodes and faces on a cut (a window side that is not a side of the box)
    are incomplete; every cell row is complete."""
    N = prob.nx
    i0, j0, k0 = org
    a = np.arange(w + 1)
    c = np.arange(w)
    gnode = lambda i, j, k: i + (N + 1) * (j + (N + 1) * k)
    K, J, I = np.meshgrid(a + k0, a + j0, a + i0, indexing="ij")
    nodes = gnode(I, J, K).ravel()
    K, J, I = np.meshgrid(c + k0, c + j0, c + i0, indexing="ij")
    cells = (I + N * (J + N * K)).ravel()
    nFx = (N + 1) * N * N
    nFy = N * (N + 1) * N
    K, J, I = np.meshgrid(c + k0, c + j0, a + i0, indexing="ij")
    fx = (I + (N + 1) * (J + N * K)).ravel()
    K, J, I = np.meshgrid(c + k0, a + j0, c + i0, indexing="ij")
    fy = (nFx + I + N * (J + (N + 1) * K)).ravel()
    K, J, I = np.meshgrid(a + k0, c + j0, c + i0, indexing="ij")
    fz = (nFx + nFy + I + N * (J + N * K)).ravel()
    faces = np.concatenate([fx, fy, fz])

    def inner(loc, lo):
        # local lattice index loc on an axis with w cells: not on a cut
        return ((loc > 0) | (lo == 0)) & ((loc < w) | (lo + w == N))
    K, J, I = np.meshgrid(a, a, a, indexing="ij")
    node_ok = (inner(I, i0) & inner(J, j0) & inner(K, k0)).ravel()
    K, J, I = np.meshgrid(c, c, a, indexing="ij")
    fx_ok = inner(I, i0).ravel()
    K, J, I = np.meshgrid(c, a, c, indexing="ij")
    fy_ok = inner(J, j0).ravel()
    K, J, I = np.meshgrid(a, c, c, indexing="ij")
    fz_ok = inner(K, k0).ravel()
    face_ok = np.concatenate([fx_ok, fy_ok, fz_ok])
    fbc = prob.face_bc[faces].copy()
    sub = mi.Problem(w, w, w, prob.coords[nodes].copy(), prob.node_fix[nodes].copy(), fbc,
                     prob.E[cells].copy(), prob.nu[cells].copy(), prob.biot[cells].copy(),
                     prob.Seps[cells].copy(), prob.mu[cells].copy(), prob.kappa[cells].copy(), prob.dt,
                     prob.traction.copy())
    nU = 3 * prob.n_nodes
    rows = np.concatenate([(3 * nodes[:, None] + np.arange(3)).ravel(), nU + cells, nU + prob.n_cells + faces])
    ok = np.concatenate([np.repeat(node_ok, 3), np.ones(len(cells), bool), face_ok])
    return sub, rows, ok


WINDOWS = [(0, 0, 0), (120, 120, 120), (60, 64, 56), (0, 64, 120), (64, 0, 64), (120, 30, 0)]


def test_layered_jittered_128_cubed():
    """The 128^3 jittered, layered workload (14,877,827 unknowns; kappa over
    six decades, E over two, S_eps = 0, dt = 0.1 s) at full size, in the
    bench's launch configuration.  Against the oracle on 8^3-cell windows
    (every complete row): A_H x for a seeded x and the right-hand side at
    1e-12, the float-float Arnoldi operator within 2^-40 of each row's sum of
    |terms|, D_s at 1e-12 where the row's B~_p and C~_pi diagonal are local to
    the window, and the residual b - A x of the mixed and FP64 solutions
    (relative to the size of its terms).  Properties at any size: both forms
    reach 1e-8, the no-allocation residual agrees, they agree with each
    other, and the solution is linear in the load."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_09603_gb300 import Solver
    prob = mi.layered_jitter_cube(128)
    wins = []
    for org in WINDOWS:
        sub, rows, ok = _window(prob, org, 8)
        Bw = oracle.assemble(sub)
        Aw = system.system_matrix(Bw)
        Btw = precond.btilde(Bw)
        dsw = precond.equilibration(Bw, Btw, precond.ctilde(Bw, Btw))
        wins.append((sub, Bw, Aw, rows, ok, dsw, system.rhs(Bw)))
    xseed = np.random.default_rng(128).standard_normal(prob.sizes[0] + prob.sizes[1] + prob.sizes[2])
    xs = {}
    for precision in (1, 0):
        s = Solver(prob)
        s.assemble_condense()
        s.setup_precond(_bench_options(precision, restart=20))
        assert s.sizes == (3 * 129 ** 3, 128 ** 3, 3 * 128 * 128 * 129)
        b = s.build_rhs()
        x, st = s.solve(b, tol=1e-8)
        assert st["converged"] and st["true_rel_residual"] <= 1.05e-8
        rn, bn = s.residual_norm_noalloc(b, x).cpu().numpy()
        assert rn / bn <= 1.1e-8
        ax = s.apply_operator(x).cpu().numpy()
        bb = b.cpu().numpy()
        xx = x.cpu().numpy()
        if precision == 1:
            y = s.apply_operator(torch.from_numpy(xseed).cuda()).cpu().numpy()
            zseed = xseed.astype(np.float32).astype(np.float64)
            yff = s.apply_operator_ff(torch.from_numpy(zseed).cuda()).cpu().numpy()
            for sub, Bw, Aw, rows, ok, dsw, bw in wins:
                err = np.abs(yff[rows] - Aw @ zseed[rows])[ok]
                assert np.all(err <= 2.0 ** -40 * (abs(Aw) @ np.abs(zseed[rows]))[ok] + 1e-300)
            ds = s.scalings()[1].cpu().numpy()
            for sub, Bw, Aw, rows, ok, dsw, bw in wins:
                ref = Aw @ xseed[rows]
                scale = np.abs(ref).max()
                assert np.abs(y[rows][ok] - ref[ok]).max() <= 1e-12 * scale
                assert np.abs(bb[rows][ok] - bw[ok]).max() <= 1e-12 * max(np.abs(bw).max(), 1e-300)
                # D_s rows whose B~_p (the cell's 8 nodes) and C~_pi diagonal
                # (the face's cells) are local: u rows of complete nodes and
                # p and pi rows of the window's interior cells and faces
                nUw, nPw, _ = Bw.sizes
                cell_ok = np.ones(nPw, bool)
                Bw_nodes_ok = ok[:nUw].reshape(-1, 3)[:, 0]
                cell_ok &= Bw_nodes_ok[Bw.mesh.cell_nodes].all(axis=1)
                fc = Bw.mesh.face_cells
                face_ok = ok[nUw + nPw:] & np.all((fc < 0) | cell_ok[np.maximum(fc, 0)], axis=1)
                dmask = np.concatenate([ok[:nUw], cell_ok, face_ok])
                assert dmask[nUw:nUw + nPw].sum() > 0 and dmask[nUw + nPw:].sum() > 0
                assert np.allclose(ds[rows][dmask], dsw[dmask], rtol=1e-12, atol=0)
            x2, _ = s.solve(s.build_rhs(None, load_scale=2.0), tol=1e-8)
            d = (x2 - 2 * x).norm() / (2 * x).norm()
            assert d.item() <= 1e-5
        for sub, Bw, Aw, rows, ok, dsw, bw in wins:
            rw = bw - Aw @ xx[rows]
            scale = np.abs(bw).max() + np.abs(Aw @ xx[rows]).max()
            assert np.abs((bb - ax)[rows][ok] - rw[ok]).max() <= 1e-12 * scale
        xs[precision] = xx
        s.close()
    diff = np.linalg.norm(xs[1] - xs[0]) / np.linalg.norm(xs[0])
    assert diff <= 1e-5, diff
