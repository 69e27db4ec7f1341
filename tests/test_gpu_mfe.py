"""The mixed formulation [u | p | q] (Eq. mfeSys with the stabilization of
Eq. stab_A) and its block-triangular preconditioner M_II^(m) (Eq. prec) on
the GPU, through the C ABI (options.formulation = 1), against the oracle's
oracle/mixed.py element by element: the operator's rows, the equilibration,
C~_p and its cell hierarchy (every level operator and Chebyshev bound), the
A_qq level, both V-cycles, M^-1, and FGMRES reaching the mixed system's
direct solution with the oracle's iteration count.

Tolerances as in test_gpu_parity.py: assembled blocks and operator applies
1e-12 relative to the largest entry of their block, multigrid levels 1e-11,
V-cycles and M^-1 1e-10, solves 1e-8 in the energy norm at a 1e-10
residual tolerance."""
import numpy as np
import pytest

import mhfp_inputs as mi
import oracle
from oracle import fgmres, mixed, precond, system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


CASES = [
    ("cantilever8", lambda: mi.cantilever_cube(8)),
    ("cantilever8_small_dt", lambda: mi.cantilever_cube(8, dt=1e-5)),
    ("ragged", lambda: mi.random_small(10, 9, 8, seed=12, jitter=0.15)),
    ("terzaghi12", lambda: mi.terzaghi_cube(12, dt=10.0)),
    ("three_levels", lambda: mi.random_small(16, 16, 16, seed=13, jitter=0.1)),
]


def _solver(prob, formulation=1, near_kernel=0, precision=0):
    from paper_2002_09603_gb300 import Solver, default_options
    opt = default_options()
    opt.formulation = formulation
    opt.near_kernel = near_kernel
    opt.precision = precision
    s = Solver(prob)
    s.assemble_condense()
    s.setup_precond(opt)
    return s


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    prob = request.param[1]()
    B = oracle.assemble(prob)
    M = mixed.assemble_mixed(B, prob.face_bc)
    pc = mixed.build_btp(M, "amg")
    s = _solver(prob)
    yield request.param[0], prob, B, M, pc, s
    s.close()


def _close(got, ref, rtol, what):
    scale = max(np.abs(ref).max(), 1e-300)
    err = np.abs(got - ref).max() / scale
    assert err <= rtol, (what, err)


def _blockwise(got, ref, sizes, rtol):
    o = 0
    for k, n in enumerate(sizes):
        _close(got[o:o + n], ref[o:o + n], rtol, ("block", k))
        o += n


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_operator_rows(case):
    name, prob, B, M, pc, s = case
    rng = np.random.default_rng(21)
    A = mixed.mixed_matrix(M)
    for _ in range(2):
        x = rng.standard_normal(s.n)
        y = s.apply_operator(_gpu(x)).cpu().numpy()
        _blockwise(y, A @ x, B.sizes, 1e-12)


def test_equilibration_and_cp_diagonal(case):
    name, prob, B, M, pc, s = case
    bt, ds = s.scalings()
    _close(bt.cpu().numpy(), pc.Cp.diagonal(), 1e-12, "diag C~_p")
    _blockwise(ds.cpu().numpy(), mixed.equilibration(M, pc.Cp), B.sizes, 1e-12)


def test_cp_hierarchy_levels(case):
    name, prob, B, M, pc, s = case
    info = s.hierarchy(1)
    assert info["levels"] == len(pc.p_levels)
    if name == "three_levels":
        assert info["levels"] == 3
    assert info["block"] == [1] * info["levels"]
    rng = np.random.default_rng(22)
    for l, lev in enumerate(pc.p_levels):
        n = lev.A.shape[0]
        assert info["points"][l] == n
        if l < len(pc.p_levels) - 1:
            assert np.isclose(info["lmax"][l], lev.lmax, rtol=1e-11), (l, info["lmax"][l], lev.lmax)
        x = rng.standard_normal(n)
        y = s.level_apply(1, l, _gpu(x)).cpu().numpy()
        _close(y, lev.A @ x, 1e-12 if l == 0 else 1e-11, ("C~_p level", l))


def test_flux_level(case):
    name, prob, B, M, pc, s = case
    info = s.hierarchy(2)
    assert info["levels"] == 1 and info["points"] == [B.sizes[2]]
    assert np.isclose(info["lmax"][0], pc.q_level.lmax, rtol=1e-11)
    x = np.random.default_rng(23).standard_normal(B.sizes[2])
    _close(s.level_apply(2, 0, _gpu(x)).cpu().numpy(), M.Aqq @ x, 1e-12, "A_qq")


def test_vcycles_and_preconditioner(case):
    name, prob, B, M, pc, s = case
    rng = np.random.default_rng(24)
    nU, nP, nF = B.sizes
    bp = rng.standard_normal(nP)
    _close(s.vcycle(1, _gpu(bp)).cpu().numpy(), precond.vcycle(pc.p_levels, bp), 1e-10, "V(C~_p)")
    bu = rng.standard_normal(nU)
    _close(s.vcycle(0, _gpu(bu)).cpu().numpy(), precond.vcycle(pc.u_levels, bu), 1e-10, "V(A_uu)")
    for _ in range(2):
        v = rng.standard_normal(s.n)
        z = s.apply_precond(_gpu(v)).cpu().numpy()
        _blockwise(z, pc.apply(v), B.sizes, 1e-10)


def test_solve_reaches_the_direct_solution(case):
    name, prob, B, M, pc, s = case
    b = s.build_rhs()
    bref = system.rhs(B)
    _blockwise(b.cpu().numpy(), bref, B.sizes, 1e-12)
    x, st = s.solve(b, tol=1e-10)
    assert st["converged"] and st["true_rel_residual"] <= 1.05e-10
    xd = mixed.solve_direct(M, bref)
    nU, nP, _ = B.sizes
    e = x.cpu().numpy() - xd

    def enorm(v):
        return np.sqrt(v[:nU] @ (B.Auu @ v[:nU]) + v[nU:nU + nP] @ (pc.Cp @ v[nU:nU + nP])
                       + v[nU + nP:] @ (M.Aqq @ v[nU + nP:]))
    assert enorm(e) <= 1e-8 * enorm(xd)
    A = mixed.mixed_matrix(M)
    _, info = fgmres.fgmres(lambda q: A @ q, pc.apply, bref, tol=1e-10, scale=mixed.equilibration(M, pc.Cp))
    assert abs(info["iters"] - st["iterations"]) <= 1, (info["iters"], st["iterations"])


def test_hybrid_only_calls_are_refused():
    from paper_2002_09603_gb300 import MhfpError
    prob = mi.random_small(4, 4, 3, seed=2)
    s = _solver(prob)
    v = _gpu(np.ones(s.n))
    for call in (lambda: s.apply_operator_t(v), lambda: s.apply_precond_t(v),
                 lambda: s.update_logk(_gpu(np.zeros(s.sizes[1]))),
                 lambda: s.residual_norm_noalloc(v, v, out=_gpu(np.zeros(2)))):
        with pytest.raises(MhfpError, match="mixed formulation"):
            call()
    s.close()
    with pytest.raises(MhfpError):
        _solver(prob, precision=1)


def test_mixed_form_at_the_table_grid_64():
    """The 1/h = 64 cantilever of Table tab:can_3 (1,884,739 unknowns,
    dt = 1e-5) in the mixed form, at full size against the oracle: every
    operator row (1e-12), D_s and C~_p's diagonal (1e-12), C~_p itself (the
    first level of its hierarchy, 1e-12), and the solution of the bench's
    configuration (FGMRES(30), tolerance 1e-6 and 1e-8) checked by the
    residual recomputed with the oracle's assembled mixed matrix.  The same
    problem in the hybrid form with M_II^(h) and M_III^(h) (the table's other
    columns): operator rows and the solutions' residuals recomputed with the
    oracle's assembled hybrid matrix."""
    prob = mi.cantilever_cube(64, dt=1e-5)
    B = oracle.assemble(prob)
    M = mixed.assemble_mixed(B, prob.face_bc)
    A = mixed.mixed_matrix(M)
    Cp = mixed.ctilde_p(M)
    from paper_2002_09603_gb300 import Solver, default_options
    opt = default_options()
    opt.formulation = 1
    opt.restart = 30
    s = Solver(prob)
    s.assemble_condense()
    s.setup_precond(opt)
    rng = np.random.default_rng(64)
    x = rng.standard_normal(s.n)
    _blockwise(s.apply_operator(_gpu(x)).cpu().numpy(), A @ x, B.sizes, 1e-12)
    bt, ds = s.scalings()
    _close(bt.cpu().numpy(), Cp.diagonal(), 1e-12, "diag C~_p")
    _blockwise(ds.cpu().numpy(), mixed.equilibration(M, Cp), B.sizes, 1e-12)
    xp = rng.standard_normal(B.sizes[1])
    _close(s.level_apply(1, 0, _gpu(xp)).cpu().numpy(), Cp @ xp, 1e-12, "C~_p")
    b = s.build_rhs()
    bref = system.rhs(B)
    _blockwise(b.cpu().numpy(), bref, B.sizes, 1e-12)
    d = ds.cpu().numpy()
    for tol in (1e-6, 1e-8):
        xs, st = s.solve(b, tol=tol)
        assert st["converged"]
        r = d * (bref - A @ xs.cpu().numpy())
        assert np.linalg.norm(r) <= 1.05 * tol * np.linalg.norm(d * bref), (tol, np.linalg.norm(r) / np.linalg.norm(d * bref))
    s.close()
    AH = system.system_matrix(B)
    for nk in (0, 1):
        opt = default_options()
        opt.near_kernel = nk
        opt.restart = 30
        s = Solver(prob)
        s.assemble_condense()
        s.setup_precond(opt)
        _blockwise(s.apply_operator(_gpu(x)).cpu().numpy(), AH @ x, B.sizes, 1e-12)
        d = s.scalings()[1].cpu().numpy()
        b = s.build_rhs()
        _blockwise(b.cpu().numpy(), bref, B.sizes, 1e-12)
        xs, st = s.solve(b, tol=1e-8)
        assert st["converged"]
        r = d * (bref - AH @ xs.cpu().numpy())
        assert np.linalg.norm(r) <= 1.05e-8 * np.linalg.norm(d * bref), (nk, np.linalg.norm(r) / np.linalg.norm(d * bref))
        s.close()


def test_mixed_form_with_rigid_body_modes_and_in_a_batch():
    """formulation = 1 combined with the rigid-body-mode displacement
    multigrid (near_kernel = 1) reaches the mixed system's direct solution,
    and mixed-form handles solved together (mhfp_solve_batch) give the same
    solutions as one at a time."""
    from paper_2002_09603_gb300 import solve_batch
    prob = mi.cantilever_cube(8, dt=1e-5)
    B = oracle.assemble(prob)
    M = mixed.assemble_mixed(B, prob.face_bc)
    bref = system.rhs(B)
    xd = mixed.solve_direct(M, bref)
    s = _solver(prob, near_kernel=1)
    assert s.hierarchy(0)["block"][1:] == [6] * (s.hierarchy(0)["levels"] - 1)
    x, st = s.solve(s.build_rhs(), tol=1e-10)
    assert st["converged"]
    assert np.linalg.norm(x.cpu().numpy() - xd) <= 1e-7 * np.linalg.norm(xd)
    s2 = _solver(mi.random_small(10, 9, 8, seed=12, jitter=0.15))
    bs = [s.build_rhs(), s2.build_rhs()]
    xs, stats, codes = solve_batch([s, s2], bs, tol=1e-10)
    assert list(codes) == [0, 0]
    for h, b, xb in zip((s, s2), bs, xs):
        x1, _ = h.solve(b, tol=1e-10)
        assert torch.equal(x1, xb)
    s.close()
    s2.close()
