"""Adjoint solve and log-permeability gradient through the C ABI, against
the FP64 oracle's transposed operator, transposed preconditioner and
discrete-adjoint gradient, and against central finite differences."""
import numpy as np
import pytest

import mhfp_inputs as mi
import oracle
from oracle import adjoint, precond, system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _iso(p):
    p.kappa = np.repeat(p.kappa[:, :1], 3, axis=1)
    return p


@pytest.fixture(scope="module", params=[0, 1], ids=["fp64", "fp32vc"])
def case(request):
    from paper_2002_09603_gb300 import Solver, default_options
    prob = _iso(mi.random_small(5, 4, 6, seed=31, jitter=0.15, dt=0.05))
    B = oracle.assemble(prob)
    pc = precond.build(B, "amg")
    opt = default_options()
    opt.precision = request.param
    s = Solver(prob)
    s.assemble_condense()
    s.setup_precond(opt)
    yield prob, B, pc, s, request.param
    s.close()


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_transposed_operator(case):
    prob, B, pc, s, _ = case
    x = np.random.default_rng(1).standard_normal(s.n)
    y = s.apply_operator_t(_cuda(x)).cpu().numpy()
    ref = system.system_matrix(B).T @ x
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()


def test_transposed_preconditioner(case):
    """M^-T from forward substitution equals the oracle's, and is the adjoint
    of M^-1: <M^-T a, b> = <a, M^-1 b> (the V-cycles are symmetric)."""
    prob, B, pc, s, prec = case
    rng = np.random.default_rng(2)
    a, b = rng.standard_normal((2, s.n))
    za = s.apply_precond_t(_cuda(a)).cpu().numpy()
    zb = s.apply_precond(_cuda(b)).cpu().numpy()
    tol = 1e-10 if prec == 0 else 1e-5
    ref = pc.apply_transpose(a)
    assert np.abs(za - ref).max() <= tol * np.abs(ref).max()
    assert abs(za @ b - a @ zb) <= tol * abs(a @ zb) * 10


def test_adjoint_solve_identity(case):
    """A^T lambda = r solved directly equals D A^-1 D^-1 r with
    D = diag(I, -I, -dt I) solved by the forward FGMRES."""
    prob, B, pc, s, _ = case
    nU, nP, nPi = B.sizes
    r = np.random.default_rng(3).standard_normal(s.n)
    r[nU + nP:][B.pi_fixed] = 0.0
    lam, st = s.adjoint_solve(_cuda(r), tol=1e-11)
    assert st["converged"]
    lam = lam.cpu().numpy()
    ref = oracle.adjoint.spla.spsolve(system.system_matrix(B).T.tocsc(), r)
    D = np.concatenate([np.ones(nU), -np.ones(nP), -B.dt * np.ones(nPi)])
    xf, _ = s.solve(_cuda(r / D), tol=1e-11)
    via = D * xf.cpu().numpy()
    for got in (lam, via):
        o = 0
        for n_ in B.sizes:
            assert np.abs(got[o:o + n_] - ref[o:o + n_]).max() <= 1e-6 * np.abs(ref[o:o + n_]).max()
            o += n_


def _targets(prob, nsteps, seed):
    q = mi.Problem(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in prob.__dict__.items()})
    q.kappa *= np.exp(np.random.default_rng(seed).uniform(-0.5, 0.5, (prob.n_cells, 1)))
    Bq = oracle.assemble(q)
    xq = adjoint.forward(Bq, nsteps)
    nU, nP, _ = Bq.sizes
    dofs = adjoint.top_uz_dofs(Bq)
    return [x[dofs] for x in xq], [x[nU:nU + nP] for x in xq]


def test_gradient_matches_oracle_and_checkpointing():
    """dJ/d ln kappa on the GPU (forward + reverse sweep through the ABI)
    equals the oracle's discrete adjoint (direct solves), also when only
    every third state is kept and segments are recomputed."""
    from paper_2002_09603_gb300.adjoint import MisfitGradient
    prob = _iso(mi.random_small(5, 4, 6, seed=31, jitter=0.15, dt=0.05))
    nsteps = 4
    targets = _targets(prob, nsteps, 5)
    B = oracle.assemble(prob)
    Jo, go, _ = adjoint.gradient(B, nsteps, adjoint.Misfit(B, *targets))
    logk = np.log(prob.kappa[:, 0])
    for k in (1, 3):
        mg = MisfitGradient(prob, nsteps, *targets, tol=1e-13, checkpoint_every=k)
        J, g = mg.value_and_grad(logk)
        g = g.cpu().numpy()
        assert np.isclose(J, Jo, rtol=1e-9)
        assert np.abs(g - go).max() <= 1e-7 * np.abs(go).max(), k


def test_gradient_central_differences_and_autograd():
    """The GPU gradient agrees with central finite differences of the GPU
    misfit (1e-5 relative on the cells with the largest sensitivities), and
    the torch.autograd.Function returns it."""
    from paper_2002_09603_gb300.adjoint import MisfitGradient, make_autograd
    prob = _iso(mi.lognormal_cube(12, seed=5, sigma=1.0, dt=0.1))
    nsteps = 4
    targets = _targets(prob, nsteps, 9)
    mg = MisfitGradient(prob, nsteps, *targets, tol=1e-14, checkpoint_every=2)
    logk = np.log(prob.kappa[:, 0])
    J, g = mg.value_and_grad(logk)
    g = g.cpu().numpy()
    h = 1e-3
    for T in np.argsort(-np.abs(g))[:5]:
        lp, lm = logk.copy(), logk.copy()
        lp[T] += h
        lm[T] -= h
        fd = (mg.value(lp) - mg.value(lm)) / (2 * h)
        assert np.isclose(g[T], fd, rtol=1e-5), (T, g[T], fd)
    f = make_autograd(mg)
    t = torch.tensor(logk, dtype=torch.float64, requires_grad=True)
    Jt = f(t)
    Jt.backward()
    assert np.isclose(Jt.item(), J, rtol=1e-12)
    assert np.allclose(t.grad.numpy(), g, rtol=1e-9, atol=1e-12 * np.abs(g).max())


def test_adjoint_workload_48_cubed():
    """The 48^3, 10-step adjoint workload (log-normal sigma 1, dt = 0.1 s,
    targets from a second seeded field): the reverse sweep converges every
    solve, and on the ten most sensitive cells the gradient agrees with
    central differences of J at h = 1e-4 to 1e-4 relative.  (J ~ 7e3 is
    known to ~4e-13 relative at a 1e-14 tolerance, so h = 1e-6 would leave
    ~1e-3 of noise even on the largest cell sensitivity.)"""
    from paper_2002_09603_gb300 import Solver
    from paper_2002_09603_gb300.adjoint import MisfitGradient
    n, nsteps = 48, 10
    prob = mi.lognormal_cube(n, seed=5, sigma=1.0, dt=0.1)
    q = mi.lognormal_cube(n, seed=55, sigma=1.0, dt=0.1)
    s = Solver(q)
    s.assemble_condense()
    s.setup_precond()
    nU, nP, _ = s.sizes
    nodes = np.arange((n + 1) ** 3)
    top = nodes[nodes // ((n + 1) ** 2) == n]
    x, uz, pp = None, [], []
    for _ in range(nsteps):
        x, _ = s.solve(s.build_rhs(x), tol=1e-13)
        xc = x.cpu().numpy()
        uz.append(xc[3 * top + 2])
        pp.append(xc[nU:nU + nP])
    s.close()
    mg = MisfitGradient(prob, nsteps, uz, pp, tol=1e-14, checkpoint_every=3)
    logk = np.log(prob.kappa[:, 0])
    J, g = mg.value_and_grad(logk)
    assert all(st["converged"] for st in mg.stats)
    g = g.cpu().numpy()
    h = 1e-4
    for T in np.argsort(-np.abs(g))[:10]:
        lp, lm = logk.copy(), logk.copy()
        lp[T] += h
        lm[T] -= h
        fd = (mg.value(lp) - mg.value(lm)) / (2 * h)
        assert np.isclose(g[T], fd, rtol=1e-4), (T, g[T], fd)


@pytest.mark.parametrize("precision", [0, 1])
def test_update_logk_in_place(precision):
    """mhfp_update_logk on a handle that has already solved (and captured its
    solve graphs) gives bit-identical operator, M^-1, solutions and iteration
    counts to the same update on a freshly set-up handle; both agree with a
    handle created from the new permeability (computed on the host) and with
    the oracle's direct solution; a non-finite log-permeability is rejected
    and leaves the handle unchanged."""
    from paper_2002_09603_gb300 import MhfpError, Solver, default_options
    from paper_2002_09603_gb300.adjoint import _with_logk
    prob = mi.random_small(6, 5, 4, seed=41, jitter=0.1, dt=0.05)
    rng = np.random.default_rng(7)
    logk = np.log(prob.kappa[:, 0]) + rng.normal(0.0, 1.0, prob.n_cells)
    opt = default_options()
    opt.precision = precision

    def handle(p):
        s = Solver(p)
        s.assemble_condense()
        s.setup_precond(opt)
        return s

    used = handle(prob)
    x0, _ = used.solve(used.build_rhs(), tol=1e-10)          # captures the solve graph
    used.adjoint_solve(used.build_rhs(), tol=1e-10)
    lmax_before = used.hierarchy(1)["lmax"]
    fresh = handle(prob)
    t = _cuda(logk)
    used.update_logk(t)
    fresh.update_logk(t)
    host = handle(_with_logk(prob, logk))
    assert used.hierarchy(1)["lmax"] != lmax_before
    assert np.allclose(used.hierarchy(1)["lmax"], host.hierarchy(1)["lmax"], rtol=1e-11)
    v = _cuda(rng.standard_normal(used.n))
    outs = {}
    for name, s in (("used", used), ("fresh", fresh), ("host", host)):
        b = s.build_rhs(x0)
        x, st = s.solve(b, tol=1e-10)
        lam, sta = s.adjoint_solve(b, tol=1e-10)
        outs[name] = dict(y=s.apply_operator(v), z=s.apply_precond(v), x=x, it=st["iterations"],
                          lam=lam, ita=sta["iterations"], ds=s.scalings()[1])
    for k in ("y", "z", "x", "lam", "ds"):
        assert torch.equal(outs["used"][k], outs["fresh"][k]), k
    assert outs["used"]["it"] == outs["fresh"]["it"] and outs["used"]["ita"] == outs["fresh"]["ita"]
    # against a handle built from the host-computed permeability (exp may
    # differ in the last bit) and the oracle
    Bq = oracle.assemble(_with_logk(prob, logk))
    yref = system.system_matrix(Bq) @ v.cpu().numpy()
    for name in ("used", "host"):
        y = outs[name]["y"].cpu().numpy()
        assert np.abs(y - yref).max() <= 1e-12 * np.abs(yref).max()
    zt = 1e-10 if precision == 0 else 1e-5
    zu, zh = outs["used"]["z"].cpu().numpy(), outs["host"]["z"].cpu().numpy()
    assert np.abs(zu - zh).max() <= zt * np.abs(zh).max()
    assert abs(outs["used"]["it"] - outs["host"]["it"]) <= 1
    nU, nP, _ = Bq.sizes
    xc = x0.cpu().numpy()
    xd = oracle.solve_direct(Bq, system.rhs(Bq, xc[:nU], xc[nU:nU + nP]))
    xu = outs["used"]["x"].cpu().numpy()
    assert np.linalg.norm(xu - xd) <= 1e-7 * np.linalg.norm(xd)
    # rejected update: nothing changes
    bad = logk.copy()
    bad[3] = np.nan
    with pytest.raises(MhfpError):
        used.update_logk(_cuda(bad))
    assert torch.equal(used.apply_operator(v), outs["used"]["y"])
    for s in (used, fresh, host):
        s.close()
