"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: FP64 operator applies and assembled blocks 1e-12 relative (to
the largest entry of the block they belong to); multigrid levels 1e-11
(their Chebyshev bounds come from power iterations summed in a different
order); full solves 1e-8 relative in the block-diagonal energy norm at a
1e-10 residual tolerance.
"""
import numpy as np
import pytest

import mhfp_inputs as mi
import oracle
from oracle import fgmres, precond, system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _prep(prob):
    from paper_2002_09603_gb300 import prepare
    return prepare(prob)


def _blockwise_close(got, ref, sizes, rtol):
    o = 0
    for n in sizes:
        g, r = got[o:o + n], ref[o:o + n]
        scale = max(np.abs(r).max(), 1e-300)
        assert np.abs(g - r).max() <= rtol * scale, (o, n, np.abs(g - r).max() / scale)
        o += n


CASES = [
    ("cube2", lambda: mi.random_small(2, 2, 2, seed=1)),
    ("odd", lambda: mi.random_small(3, 2, 5, seed=2, jitter=0.2)),
    ("jitter7", lambda: mi.random_small(7, 6, 5, seed=3, jitter=0.25)),
    ("one", lambda: mi.random_small(1, 1, 1, seed=4)),
    ("terzaghi8", lambda: mi.terzaghi_cube(8)),
    ("ragged", lambda: mi.random_small(10, 4, 7, seed=5, jitter=0.1)),
    # the 128^3 workload's physics at 16^3: jitter 0.2h, 8 layers with kappa over
    # six decades and E over two, S_eps = 0, dt = 0.1 s
    ("layered16", lambda: mi.layered_jitter_cube(16)),
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    prob = request.param[1]()
    B = oracle.assemble(prob)
    pc = precond.build(B, "amg")
    s = _prep(prob)
    yield prob, B, pc, s
    s.close()


def test_sizes(case):
    prob, B, pc, s = case
    assert s.sizes == B.sizes == prob.sizes


def test_operator_apply(case):
    prob, B, pc, s = case
    rng = np.random.default_rng(0)
    x = rng.standard_normal(s.n)
    y = s.apply_operator(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = system.system_matrix(B) @ x
    _blockwise_close(y, ref, B.sizes, 1e-12)


def test_btilde_and_scaling(case):
    prob, B, pc, s = case
    bt, ds = s.scalings()
    assert np.allclose(bt.cpu().numpy(), pc.Bt, rtol=1e-12, atol=0)
    assert np.allclose(ds.cpu().numpy(), precond.equilibration(B, pc.Bt, pc.C), rtol=1e-12, atol=0)


def test_rhs(case):
    prob, B, pc, s = case
    rng = np.random.default_rng(1)
    x = rng.standard_normal(s.n)
    nU, nP, _ = B.sizes
    got = s.build_rhs(torch.from_numpy(x).cuda(), load_scale=2.5).cpu().numpy()
    ref = system.rhs(B, x[:nU], x[nU:nU + nP], load_scale=2.5)
    _blockwise_close(got, ref, B.sizes, 1e-12)
    got0 = s.build_rhs(None).cpu().numpy()
    _blockwise_close(got0, system.rhs(B), B.sizes, 1e-12)


def _dense_of(apply, n):
    cols = []
    for j in range(n):
        e = torch.zeros(n, dtype=torch.float64, device="cuda")
        e[j] = 1.0
        cols.append(apply(e).cpu().numpy())
    return np.stack(cols, axis=1)


def test_multigrid_levels(case):
    """Every level operator: same sizes, same sparsity pattern (bit-exact),
    values within 1e-11 of the oracle's Galerkin products."""
    prob, B, pc, s = case
    for which, levels in ((0, pc.u_levels), (1, pc.pi_levels)):
        info = s.hierarchy(which)
        assert info["levels"] == len(levels)
        rng = np.random.default_rng(2)
        for l, lev in enumerate(levels):
            n = lev.A.shape[0]
            assert info["points"][l] * info["block"][l] == n
            if l < len(levels) - 1:
                assert np.isclose(info["lmax"][l], lev.lmax, rtol=1e-11)
            x = rng.standard_normal(n)
            y = s.level_apply(which, l, torch.from_numpy(x).cuda()).cpu().numpy()
            ref = lev.A @ x
            assert np.abs(y - ref).max() <= 1e-11 * np.abs(ref).max(), (which, l)
            if n <= 700:
                D = _dense_of(lambda e: s.level_apply(which, l, e), n)
                R = lev.A.toarray()
                # same sparsity pattern up to entries that cancel to rounding
                # noise on one side (1e-12 of the level's largest entry)
                noise = 1e-12 * np.abs(R).max()
                assert np.all(R[np.abs(D) > noise] != 0) and np.all(D[np.abs(R) > noise] != 0), (which, l)
                assert np.abs(D - R).max() <= 1e-11 * np.abs(R).max()


def test_vcycles_and_preconditioner(case):
    prob, B, pc, s = case
    rng = np.random.default_rng(3)
    nU, nP, nPi = B.sizes
    bu, bpi = rng.standard_normal(nU), rng.standard_normal(nPi)
    xu = s.vcycle(0, torch.from_numpy(bu).cuda()).cpu().numpy()
    xpi = s.vcycle(1, torch.from_numpy(bpi).cuda()).cpu().numpy()
    ru, rpi = precond.vcycle(pc.u_levels, bu), precond.vcycle(pc.pi_levels, bpi)
    assert np.abs(xu - ru).max() <= 1e-10 * np.abs(ru).max()
    assert np.abs(xpi - rpi).max() <= 1e-10 * np.abs(rpi).max()
    v = rng.standard_normal(s.n)
    z = s.apply_precond(torch.from_numpy(v).cuda()).cpu().numpy()
    _blockwise_close(z, pc.apply(v), B.sizes, 1e-10)


def _energy(B, pc, v):
    nU, nP, _ = B.sizes
    return np.sqrt(v[:nU] @ (B.Auu @ v[:nU]) + v[nU:nU + nP] @ (pc.Bt * v[nU:nU + nP])
                   + v[nU + nP:] @ (pc.C @ v[nU + nP:]))


def test_solve_matches_direct_solution(case):
    prob, B, pc, s = case
    rng = np.random.default_rng(4)
    nU, nP, _ = B.sizes
    u0 = rng.standard_normal(nU) * 1e-5
    u0[B.u_fixed] = 0
    xprev = np.concatenate([u0, rng.standard_normal(nP), np.zeros(B.sizes[2])])
    b = s.build_rhs(torch.from_numpy(xprev).cuda())
    x, st = s.solve(b, tol=1e-10)
    x = x.cpu().numpy()
    bref = system.rhs(B, u0, xprev[nU:nU + nP])
    xd = oracle.solve_direct(B, bref)
    assert st["converged"] and st["true_rel_residual"] <= 1.05e-10
    assert _energy(B, pc, x - xd) <= 1e-8 * _energy(B, pc, xd)
    # same algorithm in the oracle: same iteration count up to rounding
    A = system.system_matrix(B)
    sc = precond.equilibration(B, pc.Bt, pc.C)
    _, info = fgmres.fgmres(lambda v: A @ v, pc.apply, bref, tol=1e-10, scale=sc)
    assert abs(info["iters"] - st["iterations"]) <= 1, (info["iters"], st["iterations"])


def test_time_steps_terzaghi_against_oracle():
    """Three backward-Euler steps of the consolidation column: the CUDA
    solver, chained through mhfp_build_rhs, tracks the oracle's direct
    solves step by step."""
    prob = mi.terzaghi_cube(6, dt=50.0)
    B = oracle.assemble(prob)
    pc = precond.build(B, "amg")
    xs, _ = oracle.time_steps(prob, 3, kind="direct")
    s = _prep(prob)
    x = None
    for k in range(3):
        b = s.build_rhs(x)
        x, st = s.solve(b, tol=1e-12)
        e = x.cpu().numpy() - xs[k]
        assert _energy(B, pc, e) <= 1e-8 * _energy(B, pc, xs[k]), k
    s.close()


def test_not_converged_and_nonfinite():
    from paper_2002_09603_gb300 import MhfpError, default_options, Solver
    prob = mi.random_small(5, 4, 4, seed=9)
    opt = default_options()
    opt.maxit = 2
    s = Solver(prob)
    s.assemble_condense()
    s.setup_precond(opt)
    b = s.build_rhs()
    x, st = s.solve(b, tol=1e-12, raise_not_converged=False)
    assert st["iterations"] == 2 and not st["converged"]
    with pytest.raises(MhfpError) as ei:
        s.solve(b, tol=1e-12)
    assert ei.value.status == 5
    bad = b.clone()
    bad[3] = float("nan")
    with pytest.raises(MhfpError) as ei:
        s.solve(bad, tol=1e-8)
    assert ei.value.status == 6
    with pytest.raises(MhfpError) as ei:
        s.solve(b, tol=0.0)
    assert ei.value.status == 1
    s.close()


def test_inverted_element_is_rejected():
    from paper_2002_09603_gb300 import MhfpError, Solver
    prob = mi.random_small(2, 2, 2, seed=1)
    c = prob.coords.copy()
    c[13] = c[13] + np.array([0.9, 0.9, 0.9])   # the centre node through the far corner
    prob.coords = c
    s = Solver(prob)
    with pytest.raises(MhfpError) as ei:
        s.assemble_condense()
    assert ei.value.status == 2
    s.close()


def test_call_order_is_enforced():
    from paper_2002_09603_gb300 import MhfpError, Solver
    s = Solver(mi.random_small(2, 2, 2, seed=1))
    b = s.empty()
    with pytest.raises(MhfpError) as ei:
        s.solve(b)
    assert ei.value.status == 8
    s.close()


# ------------------------------------------------------------ FP32 V-cycles
FP32_CASES = [c for c in CASES if c[0] in ("odd", "jitter7", "terzaghi8", "ragged", "layered16")]


@pytest.fixture(scope="module", params=FP32_CASES, ids=[c[0] for c in FP32_CASES])
def case32(request):
    from paper_2002_09603_gb300 import Solver, default_options
    prob = request.param[1]()
    B = oracle.assemble(prob)
    pc = precond.build(B, "amg")
    opt = default_options()
    opt.precision = 1
    s = Solver(prob)
    s.assemble_condense()
    s.setup_precond(opt)
    yield prob, B, pc, s
    s.close()


def test_fp32_preconditioner_matches_fp64_oracle(case32):
    """The mixed-precision M^-1 (FP32 V-cycles and Schur steps, FP64 coarsest
    solve) agrees with the oracle's FP64 M^-1 to FP32 accuracy: 1e-5 of each
    block's largest entry (a few hundred FP32 units in the last place after
    two V-cycles of Chebyshev(2) sweeps)."""
    prob, B, pc, s = case32
    rng = np.random.default_rng(5)
    v = rng.standard_normal(s.n)
    z = s.apply_precond(torch.from_numpy(v).cuda()).cpu().numpy()
    _blockwise_close(z, pc.apply(v), B.sizes, 1e-5)


def test_fp32_solve_reaches_fp64_accuracy(case32):
    """FGMRES is flexible, so the FP32 preconditioner does not limit the
    attainable accuracy: the same 1e-10 residual and 1e-8 energy-norm error
    as the FP64 solve, in at most a few more iterations."""
    prob, B, pc, s = case32
    b = s.build_rhs()
    x, st = s.solve(b, tol=1e-10)
    xd = oracle.solve_direct(B, system.rhs(B))
    assert st["converged"] and st["true_rel_residual"] <= 1.05e-10
    assert _energy(B, pc, x.cpu().numpy() - xd) <= 1e-8 * _energy(B, pc, xd)
    A = system.system_matrix(B)
    sc = precond.equilibration(B, pc.Bt, pc.C)
    _, info = fgmres.fgmres(lambda v: A @ v, pc.apply, system.rhs(B), tol=1e-10, scale=sc)
    assert st["iterations"] <= info["iters"] + 3, (st["iterations"], info["iters"])


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_matches_direct_launches(precision):
    """Direct launches (0), per-step graph replays (1) and the device-driven
    whole-solve graph (2, WHILE/IF conditional nodes) run the same kernels in
    the same order: identical iterates, bit for bit, over several restarts
    and across two solves (graphs reused)."""
    from paper_2002_09603_gb300 import Solver, default_options
    prob = mi.random_small(7, 6, 5, seed=3, jitter=0.25)
    xs = {}
    for graphs in (0, 1, 2):
        opt = default_options()
        opt.precision = precision
        opt.graphs = graphs
        opt.autotune = 0  # same launch schedule in both runs
        opt.restart = 8
        s = Solver(prob)
        s.assemble_condense()
        s.setup_precond(opt)
        b = s.build_rhs()
        x1, st1 = s.solve(b, tol=1e-10)
        x2, st2 = s.solve(s.build_rhs(x1), tol=1e-10)
        xs[graphs] = (x1.cpu().numpy(), x2.cpu().numpy(), st1["iterations"], st2["iterations"])
        s.close()
    for g in (1, 2):
        assert xs[0][2:] == xs[g][2:]
        assert np.array_equal(xs[0][0], xs[g][0]) and np.array_equal(xs[0][1], xs[g][1])


def test_device_driven_solve_stops_on_maxit_and_nonfinite():
    """The whole-solve graph ends its WHILE loop on maxit (reporting
    not-converged with the last iterate) and on a NaN right-hand side."""
    from paper_2002_09603_gb300 import MhfpError, Solver, default_options
    prob = mi.random_small(5, 4, 4, seed=9)
    opt = default_options()
    opt.graphs = 2
    opt.maxit = 5
    opt.restart = 3
    s = Solver(prob)
    s.assemble_condense()
    s.setup_precond(opt)
    b = s.build_rhs()
    x, st = s.solve(b, tol=1e-12, raise_not_converged=False)
    assert st["iterations"] == 5 and not st["converged"] and st["restarts"] == 2
    assert torch.isfinite(x).all()
    bad = b.clone()
    bad[7] = float("nan")
    with pytest.raises(MhfpError) as ei:
        s.solve(bad, tol=1e-8)
    assert ei.value.status == 6
    s.close()


def test_batch_solve_matches_individual_solves():
    """mhfp_solve_batch over handles of uneven size, each on its own stream,
    gives the same iterates as solving each handle alone (same kernels, same
    order per handle), for every load of the batched workload."""
    from paper_2002_09603_gb300 import solve_batch
    from paper_2002_09603_gb300.batch import prepare_batch
    probs = [mi.lognormal_cube(n, seed=s, sigma=1.5) for n, s in ((6, 1), (11, 2), (9, 3), (14, 4))]
    solvers = prepare_batch(probs, precision=1, restart=12)
    for scale in (0.5, 2.0):
        rhs = [s.build_rhs(None, load_scale=scale) for s in solvers]
        torch.cuda.synchronize()
        alone = []
        for s, b in zip(solvers, rhs):
            x, st = s.solve(b, tol=1e-9)
            s.stream.synchronize()
            alone.append((x.cpu().numpy(), st["iterations"]))
        xs, stats, codes = solve_batch(solvers, rhs, tol=1e-9)
        torch.cuda.synchronize()
        assert codes == [0] * len(solvers)
        for (xa, ia), xb, st in zip(alone, xs, stats):
            assert st["iterations"] == ia and st["converged"]
            assert np.array_equal(xa, xb.cpu().numpy())
    for s in solvers:
        s.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["jitter7", "ragged", "layered16"])
def test_single_pass_gram_schmidt_reaches_the_same_solution(name, precision):
    """reorth = 0 (one classical Gram-Schmidt pass per Arnoldi step, no
    reorthogonalisation) reaches the same 1e-10 true residual and 1e-8
    energy-norm error against the oracle's direct solution as the DGKS form,
    in at most two more iterations."""
    from paper_2002_09603_gb300 import Solver, default_options
    prob = dict(CASES)[name]()
    B = oracle.assemble(prob)
    pc = precond.build(B, "amg")
    xd = oracle.solve_direct(B, system.rhs(B))
    its = {}
    for reorth in (1, 0):
        opt = default_options()
        opt.precision = precision
        opt.restart = 12
        opt.reorth = reorth
        s = Solver(prob)
        s.assemble_condense()
        s.setup_precond(opt)
        x, st = s.solve(s.build_rhs(), tol=1e-10)
        assert st["converged"] and st["true_rel_residual"] <= 1.05e-10
        assert _energy(B, pc, x.cpu().numpy() - xd) <= 1e-8 * _energy(B, pc, xd)
        its[reorth] = st["iterations"]
        s.close()
    assert its[0] <= its[1] + 2, its


def test_invalid_reorth_is_rejected():
    from paper_2002_09603_gb300 import MhfpError, Solver, default_options
    opt = default_options()
    opt.reorth = 2
    s = Solver(mi.random_small(2, 2, 2, seed=1))
    s.assemble_condense()
    with pytest.raises(MhfpError):
        s.setup_precond(opt)
    s.close()


def test_timing_classes_nest():
    """With timing on, every class records one interval per event: the
    preconditioner apply (3) holds both V-cycles (4, 5), and the displacement
    V-cycle holds the timed finest-level sweeps (0); the Arnoldi step's
    float-float operator (6) runs once per iteration, the FP64 operator (1)
    for the residual of each restart cycle and at exit; class 7 does not
    exist."""
    from paper_2002_09603_gb300 import MhfpError, Solver, default_options
    opt = default_options()
    opt.precision = 1
    opt.restart = 6
    s = Solver(mi.random_small(7, 6, 5, seed=3, jitter=0.25))
    s.assemble_condense()
    s.setup_precond(opt)
    b = s.build_rhs()
    s.timing(True)
    x, st = s.solve(b, tol=1e-8)
    r = [s.timing_read(k) for k in range(7)]
    s.timing(False)
    its = st["iterations"]
    assert r[3]["launches"] == its and r[4]["launches"] == its and r[5]["launches"] == its
    assert r[6]["launches"] == its and r[2]["launches"] == its
    assert 1 <= r[1]["launches"] <= st["restarts"] + 3
    # Chebyshev(2): the first pre-smoothing sweep starts from zero and is not
    # a stencil sweep; the second and both post-smoothing sweeps are timed
    assert r[0]["launches"] == 3 * its
    assert all(t["total_ms"] > 0 for t in r)
    assert r[3]["total_ms"] >= r[4]["total_ms"] + r[5]["total_ms"]
    assert r[4]["total_ms"] >= r[0]["total_ms"]
    with pytest.raises(MhfpError):
        s.timing_read(7)
    s.close()


def test_coarse_limit_512_against_oracle():
    """The benchmark's coarsening limit (coarse_max = 512): on a 16^3 mesh
    both hierarchies stop at 6^3 = 216 lattice points (with the default 125
    they coarsen once more), whose dense inverse (648 and 216 unknowns) is
    built on the GPU by Gauss-Jordan elimination.
    The hierarchy, both V-cycles and M^-1 match the oracle built with the same
    limit, and FGMRES reaches the direct solution."""
    from paper_2002_09603_gb300 import Solver, default_options
    prob = mi.random_small(16, 16, 16, seed=6, jitter=0.1)
    B = oracle.assemble(prob)
    pc = precond.build(B, "amg", coarse_max=512)
    assert [lv.dims for lv in pc.u_levels][-1] == (6, 6, 6)
    xd = oracle.solve_direct(B, system.rhs(B))
    rng = np.random.default_rng(8)
    nU, nP, nPi = B.sizes
    for precision in (0, 1):
        opt = default_options()
        opt.coarse_max = 512
        opt.precision = precision
        s = Solver(prob)
        s.assemble_condense()
        s.setup_precond(opt)
        assert s.hierarchy(0)["points"] == [17 ** 3, 216]
        assert s.hierarchy(1)["points"] == [B.mesh.n_faces, 16 ** 3, 216]
        v = rng.standard_normal(s.n)
        z = s.apply_precond(torch.from_numpy(v).cuda()).cpu().numpy()
        if precision == 0:
            bu, bpi = rng.standard_normal(nU), rng.standard_normal(nPi)
            xu = s.vcycle(0, torch.from_numpy(bu).cuda()).cpu().numpy()
            xpi = s.vcycle(1, torch.from_numpy(bpi).cuda()).cpu().numpy()
            ru, rpi = precond.vcycle(pc.u_levels, bu), precond.vcycle(pc.pi_levels, bpi)
            assert np.abs(xu - ru).max() <= 1e-10 * np.abs(ru).max()
            assert np.abs(xpi - rpi).max() <= 1e-10 * np.abs(rpi).max()
            _blockwise_close(z, pc.apply(v), B.sizes, 1e-10)
        else:
            _blockwise_close(z, pc.apply(v), B.sizes, 1e-5)
        x, st = s.solve(s.build_rhs(), tol=1e-10)
        assert st["converged"] and st["true_rel_residual"] <= 1.05e-10
        assert _energy(B, pc, x.cpu().numpy() - xd) <= 1e-8 * _energy(B, pc, xd)
        s.close()


# --------------------------------------------- every launch schedule, forced
SCHED_CASE = {}


def _sched_case():
    """16^3 jittered heterogeneous box: the displacement hierarchy has a
    coarse 6^3 lattice level with sweeps (3x3 blocks, 27-point stencil), the
    interface-pressure one a 16^3 cell level (25-point stencil) and a 6^3
    level (125-point stencil), so every coarse-sweep kernel kind runs."""
    if not SCHED_CASE:
        prob = mi.random_small(16, 16, 16, seed=31, jitter=0.15)
        B = oracle.assemble(prob)
        pc = precond.build(B, "amg")
        assert [lv.dims for lv in pc.u_levels] == [(17, 17, 17), (6, 6, 6), (2, 2, 2)]
        assert [lv.dims for lv in pc.pi_levels][1:] == [(16, 16, 16), (6, 6, 6), (2, 2, 2)]
        SCHED_CASE.update(prob=prob, B=B, pc=pc)
    return SCHED_CASE["prob"], SCHED_CASE["B"], SCHED_CASE["pc"]


@pytest.mark.parametrize("precision,schedule,fine_blocks",
                         [(0, 1, 0), (0, 4, 0), (0, 8, 0), (0, 16, 0),
                          (1, 1, 6), (1, 4, 8), (1, 8, 6), (1, 16, 8), (1, 8, 4)])
def test_forced_schedules_match_oracle(precision, schedule, fine_blocks):
    """Each launch schedule of the coarse-level sweeps and residuals (one
    point per thread, or the stencil offsets split over 4, 8 or 16 warps) and
    each occupancy variant of the finest FP32 displacement sweep, forced
    through mhfp_options, gives the oracle's V-cycles and M^-1 element by
    element: 1e-10 in FP64, 1e-5 in FP32 (relative to the largest entry)."""
    from paper_2002_09603_gb300 import Solver, default_options
    prob, B, pc = _sched_case()
    opt = default_options()
    opt.precision = precision
    opt.schedule = schedule
    opt.fine_blocks = fine_blocks
    s = Solver(prob)
    s.assemble_condense()
    s.setup_precond(opt)
    hu, hpi = s.hierarchy(0), s.hierarchy(1)
    assert hu["schedule"][1] == schedule and hpi["schedule"][1:3] == [schedule, schedule]
    if precision == 1:
        assert hu["schedule"][0] == fine_blocks
    tol = 1e-10 if precision == 0 else 1e-5
    rng = np.random.default_rng(40 + schedule)
    nU, nP, nPi = B.sizes
    bu, bpi = rng.standard_normal(nU), rng.standard_normal(nPi)
    xu = s.vcycle(0, torch.from_numpy(bu).cuda()).cpu().numpy()
    xpi = s.vcycle(1, torch.from_numpy(bpi).cuda()).cpu().numpy()
    ru, rpi = precond.vcycle(pc.u_levels, bu), precond.vcycle(pc.pi_levels, bpi)
    assert np.abs(xu - ru).max() <= tol * np.abs(ru).max()
    assert np.abs(xpi - rpi).max() <= tol * np.abs(rpi).max()
    v = rng.standard_normal(s.n)
    z = s.apply_precond(torch.from_numpy(v).cuda()).cpu().numpy()
    _blockwise_close(z, pc.apply(v), B.sizes, tol)
    s.close()


def test_invalid_schedule_options_are_rejected():
    from paper_2002_09603_gb300 import MhfpError, Solver, default_options
    prob = mi.random_small(3, 3, 3, seed=2)
    for field, value in (("schedule", 3), ("schedule", 32), ("fine_blocks", 3), ("fine_blocks", 9)):
        opt = default_options()
        setattr(opt, field, value)
        s = Solver(prob)
        s.assemble_condense()
        with pytest.raises(MhfpError):
            s.setup_precond(opt)
        s.close()


@pytest.mark.parametrize("dims", [(16, 16, 16), (13, 9, 21)])
def test_bulk_copy_sweep_matches_the_thread_per_node_sweep(dims):
    """Every variant of the finest FP32 displacement sweep sums the same
    products in the same order as the one-node-per-thread kernel with 8
    blocks per SM: the bulk-copy form (fine_blocks = 4: persistent CTAs,
    stored rows streamed through shared memory behind mbarriers), two slots
    per iteration (5) and the 6- and 7-block variants.  The V-cycle, M^-1 and
    a whole solve agree to FP32 rounding, on meshes of many node blocks with
    a ragged last block."""
    from paper_2002_09603_gb300 import Solver, default_options
    prob = mi.random_small(*dims, seed=33, jitter=0.1)
    out = {}
    for fb in (8, 4, 5, 6, 7):
        opt = default_options()
        opt.precision = 1
        opt.fine_blocks = fb
        s = Solver(prob)
        s.assemble_condense()
        s.setup_precond(opt)
        assert s.hierarchy(0)["schedule"][0] == fb
        rng = np.random.default_rng(9)
        bu = torch.from_numpy(rng.standard_normal(s.sizes[0])).cuda()
        v = torch.from_numpy(rng.standard_normal(s.n)).cuda()
        x, st = s.solve(s.build_rhs(), tol=1e-10)
        out[fb] = (s.vcycle(0, bu), s.apply_precond(v), x, st["iterations"])
        s.close()
    for fb in (4, 5, 6, 7):
        for k in range(3):
            a, b = out[8][k], out[fb][k]
            assert (a - b).abs().max().item() <= 1e-6 * a.abs().max().item(), (fb, k)
        assert out[8][3] == out[fb][3]


@pytest.mark.parametrize("degree", [1, 3])
def test_chebyshev_degree_matches_oracle(degree):
    """The smoother degree is an option (the set-up autotuner may pick 1, 2
    or 3): both V-cycles at degree 1 and 3 against the oracle's (1e-10)."""
    from paper_2002_09603_gb300 import Solver, default_options
    prob, B, pc = _sched_case()
    opt = default_options()
    opt.cheb_degree = degree
    s = Solver(prob)
    s.assemble_condense()
    s.setup_precond(opt)
    assert s.hierarchy(0)["cheb_degree"] == degree
    rng = np.random.default_rng(50 + degree)
    nU, nP, nPi = B.sizes
    bu, bpi = rng.standard_normal(nU), rng.standard_normal(nPi)
    xu = s.vcycle(0, torch.from_numpy(bu).cuda()).cpu().numpy()
    xpi = s.vcycle(1, torch.from_numpy(bpi).cuda()).cpu().numpy()
    ru = precond.vcycle(pc.u_levels, bu, degree=degree)
    rpi = precond.vcycle(pc.pi_levels, bpi, degree=degree)
    assert np.abs(xu - ru).max() <= 1e-10 * np.abs(ru).max()
    assert np.abs(xpi - rpi).max() <= 1e-10 * np.abs(rpi).max()
    s.close()


def test_chebyshev_degree_autotuner():
    """cheb_degree = 0: the set-up solves the step's load with degrees 1-3
    and keeps the fastest; the chosen handle still reaches the direct
    solution."""
    from paper_2002_09603_gb300 import MhfpError, Solver, default_options
    prob = mi.random_small(9, 8, 7, seed=35, jitter=0.1)
    opt = default_options()
    opt.cheb_degree = 0
    s = Solver(prob)
    s.assemble_condense()
    s.setup_precond(opt)
    assert s.hierarchy(0)["cheb_degree"] in (1, 2, 3)
    B = oracle.assemble(prob)
    xd = oracle.solve_direct(B, system.rhs(B))
    x, st = s.solve(s.build_rhs(), tol=1e-10)
    assert st["converged"] and np.linalg.norm(x.cpu().numpy() - xd) <= 1e-7 * np.linalg.norm(xd)
    s.close()
    opt.autotune = 0
    s = Solver(prob)
    s.assemble_condense()
    with pytest.raises(MhfpError):
        s.setup_precond(opt)
    s.close()


@pytest.mark.parametrize("dims,smooth", [((16, 16, 16), False), ((13, 9, 21), False), ((16, 16, 16), True)])
def test_float_float_arnoldi_operator(dims, smooth):
    """The mixed-precision Arnoldi step's operator (float-float arithmetic
    from z in FP32): every row within 2^-40 of the sum of its |terms| (|A| |z|
    row by row, from the oracle's matrix: the float-float bound is about
    2^-44 of it), also for a smooth z whose displacement rows cancel."""
    from paper_2002_09603_gb300 import Solver, default_options
    prob = mi.random_small(*dims, seed=41, jitter=0.1)
    B = oracle.assemble(prob)
    A = system.system_matrix(B)
    opt = default_options()
    opt.precision = 1
    s = Solver(prob)
    s.assemble_condense()
    s.setup_precond(opt)
    rng = np.random.default_rng(12)
    nU, nP, nPi = B.sizes
    if smooth:
        xyz = B.mesh.coords
        zu = np.stack([np.sin(xyz[:, 0] + 2 * xyz[:, 1]), np.cos(xyz[:, 2]), xyz[:, 0] * xyz[:, 1]], axis=1).ravel()
        z = np.concatenate([zu, np.ones(nP), np.ones(nPi)])
    else:
        z = rng.standard_normal(s.n)
    z = z.astype(np.float32).astype(np.float64)  # the Arnoldi step's z is FP32-exact
    zt = torch.from_numpy(z).cuda()
    yff = s.apply_operator_ff(zt).cpu().numpy()
    y64 = s.apply_operator(zt).cpu().numpy()
    ref = A @ z
    bound = 2.0 ** -40 * (abs(A) @ np.abs(z))
    err = np.abs(yff - ref)
    assert np.all(err <= bound + 1e-300), [(o, n, float((err[o:o + n] / (bound[o:o + n] + 1e-300)).max()))
                                           for o, n in ((0, nU), (nU, nP), (nU + nP, nPi))]
    assert np.abs(y64 - ref).max() <= 1e-12 * np.abs(ref).max()
    s.close()
