"""Parity on the benchmark workload at its full size (64^3, 1,884,739
unknowns), in the launch configuration bench.py times (FP32 V-cycles inside
FP64 FGMRES(12), coarsening limit 512, graphs, autotuned schedules).

The oracle assembles the whole 64^3 system (about 1.5 min on the host) and
checks, element by element, A_H x for a seeded x, then the GPU solution's
equilibrated residual recomputed with the oracle's operator, and a property
that holds at any size: with S_eps = 0 and a diffusion length sqrt(c_v dt)
far below h, one step leaves the column undrained below the drained top, so
p = sigma / b = 1 there."""
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


def test_layered_jittered_128_cubed():
    """The 128^3 jittered, layered workload (14,877,827 unknowns; kappa over
    six decades, E over two, S_eps = 0, dt = 0.1 s) at full size: the mixed
    and the FP64 solves both reach 1e-8, agree with each other, and the
    solution is linear in the load (properties that hold at any size)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_09603_gb300 import Solver, default_options
    prob = mi.layered_jitter_cube(128)
    xs = {}
    for precision in (1, 0):
        opt = default_options()
        opt.precision = precision
        opt.restart = 20
        opt.coarse_max = 512
        opt.reorth = 0
        s = Solver(prob)
        s.assemble_condense()
        s.setup_precond(opt)
        assert s.sizes == (3 * 129 ** 3, 128 ** 3, 3 * 128 * 128 * 129)
        b = s.build_rhs()
        x, st = s.solve(b, tol=1e-8)
        assert st["converged"] and st["true_rel_residual"] <= 1.05e-8
        rn, bn = s.residual_norm_noalloc(b, x).cpu().numpy()
        assert rn / bn <= 1.1e-8
        if precision == 1:
            x2, st2 = s.solve(s.build_rhs(None, load_scale=2.0), tol=1e-8)
            d = (x2 - 2 * x).norm() / (2 * x).norm()
            assert d.item() <= 1e-5
        xs[precision] = x.cpu().numpy()
        s.close()
    diff = np.linalg.norm(xs[1] - xs[0]) / np.linalg.norm(xs[0])
    assert diff <= 1e-5, diff
