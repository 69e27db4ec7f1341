"""All instances x all loads of the batched workload in one CUDA graph launch
(mhfp_batch_*), against single solves of the same handles (the same kernels
in the same order, so bit-identical results and iteration counts) and the
oracle's direct solutions; repeated launches give the same answer; a
permeability update makes the batch stale."""
import numpy as np
import pytest

import mhfp_inputs as mi
import oracle
from oracle import precond, system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _instances():
    # uneven sizes, each with its own log-normal field (the batched
    # workload's recipe at sizes the oracle solves directly)
    return [mi.lognormal_cube(n, seed=40 + n, sigma=1.5, dt=1e-3) for n in (3, 5, 8, 6, 10, 4)]


@pytest.mark.parametrize("precision", [0, 1])
def test_one_launch_matches_single_solves_and_the_oracle(precision):
    from paper_2002_09603_gb300 import MhfpError
    from paper_2002_09603_gb300.batch import LoadBatch, prepare_batch
    probs = _instances()
    solvers = prepare_batch(probs, precision=precision, restart=12, reorth=1)
    lb = LoadBatch(solvers, mi.LOAD_SCALES, tol=1e-10)
    xs, stats, codes = lb.run()
    assert codes == [0] * len(xs)
    first = [x.clone() for x in xs]
    xs2, stats2, codes2 = lb.run()
    assert all(torch.equal(a, b) for a, b in zip(first, xs2))
    k = 0
    for s, prob in zip(solvers, probs):
        B = oracle.assemble(prob)
        pc = precond.build(B, "amg")
        nU, nP, _ = B.sizes
        for scale in mi.LOAD_SCALES:
            x1, st1 = s.solve(lb.rhs[k], tol=1e-10)
            assert torch.equal(x1, first[k]), (prob.nx, scale)
            assert st1["iterations"] == stats[k]["iterations"]
            xd = oracle.solve_direct(B, system.rhs(B, load_scale=scale))
            e = first[k].cpu().numpy() - xd

            def en(v):
                return np.sqrt(v[:nU] @ (B.Auu @ v[:nU]) + v[nU:nU + nP] @ (pc.Bt * v[nU:nU + nP])
                               + v[nU + nP:] @ (pc.C @ v[nU + nP:]))
            assert en(e) <= 1e-8 * en(xd)
            k += 1
    # a permeability update on one handle makes the batch stale
    s0 = solvers[0]
    s0.update_logk(torch.as_tensor(np.log(probs[0].kappa[:, 0]), device=s0.device))
    with pytest.raises(MhfpError):
        lb.batch.run()
    lb.close()
    for s in solvers:
        s.close()


@pytest.mark.parametrize("lanes,fine_blocks,precision", [(4, 0, 1), (3, 0, 1), (4, 4, 1), (4, 0, 0)])
def test_lockstep_loads_match_single_solves_and_the_oracle(lanes, fine_blocks, precision):
    """The loads of each instance solved in lockstep (mhfp_batch_create_lanes:
    every kernel launched once for a set of right-hand sides): each member's
    solution and statistics bit-identical to the single solve of the same
    right-hand side on the same handle, and each solution against the
    oracle's direct solution (energy norm).  The right-hand sides of a set
    differ in their previous state as well as in the load, so members stop
    at different iterations, and one is zero (stops before the first cycle);
    with lanes = 3 the fourth load of an instance is a set of its own, which
    runs as a single solve; fine_blocks = 4 forces the bulk-copy finest sweep;
    precision 0 is the FP64-throughout solve.
    The sets run fewer kernels than the same solves one after another."""
    from paper_2002_09603_gb300 import launch_count
    from paper_2002_09603_gb300._lib import Batch
    from paper_2002_09603_gb300.batch import prepare_batch
    probs = _instances()
    solvers = prepare_batch(probs, precision=precision, restart=12, reorth=1, fine_blocks=fine_blocks)
    rng = np.random.default_rng(11)
    entries, rhs, out, host = [], [], [], []
    for i, (s, prob) in enumerate(zip(solvers, probs)):
        nU, nP, nPi = s.sizes
        for q, scale in enumerate(mi.LOAD_SCALES):
            if i == 2 and q == 1:
                xp, scale = None, 0.0  # b = 0
            elif q == 0:
                xp = None
            else:  # a seeded previous state [u | p | pi]
                xp = np.concatenate([1e-4 * q * rng.standard_normal(nU), rng.standard_normal(nP + nPi)])
            b = s.build_rhs(None if xp is None else torch.as_tensor(xp, device=s.device), load_scale=scale)
            entries.append(s)
            rhs.append(b)
            out.append(s.empty())
            host.append((prob, xp, scale))
    for s in solvers:
        s.stream.synchronize()
    lbatch = Batch(entries, rhs, out, tol=1e-10, lanes=lanes)
    plain = Batch(entries, rhs, [s.empty() for s in entries], tol=1e-10)
    torch.cuda.synchronize()
    l0 = launch_count()
    stats, codes = lbatch.run()
    k_lanes = launch_count() - l0
    assert codes == [0] * len(entries)
    first = [x.clone() for x in out]
    stats2, _ = lbatch.run()
    assert all(torch.equal(a, b) for a, b in zip(first, out))
    l1 = launch_count()
    pstats, pcodes = plain.run()
    k_plain = launch_count() - l1
    assert pcodes == [0] * len(entries)
    assert all(torch.equal(a, b) for a, b in zip(first, plain.out))
    assert k_lanes < k_plain, (k_lanes, k_plain)
    per_set = {}
    cache = {}
    for k, (s, (prob, xp, scale)) in enumerate(zip(entries, host)):
        x1, st1 = s.solve(rhs[k], tol=1e-10)
        assert torch.equal(x1, first[k]), (prob.nx, k)
        for key in ("iterations", "restarts", "converged", "true_rel_residual", "rel_residual"):
            assert st1[key] == stats[k][key] == pstats[k][key], (key, st1[key], stats[k][key], pstats[k][key])
        per_set.setdefault((id(s), (k % len(mi.LOAD_SCALES)) // lanes), []).append(stats[k]["iterations"])
        if id(prob) not in cache:
            B = oracle.assemble(prob)
            cache[id(prob)] = (B, precond.build(B, "amg"))
        B, pc = cache[id(prob)]
        nU, nP, _ = B.sizes
        bo = system.rhs(B, None if xp is None else xp[:nU], None if xp is None else xp[nU:nU + nP],
                        load_scale=scale)
        xd = oracle.solve_direct(B, bo)
        e = first[k].cpu().numpy() - xd

        def en(v):
            return np.sqrt(v[:nU] @ (B.Auu @ v[:nU]) + v[nU:nU + nP] @ (pc.Bt * v[nU:nU + nP])
                           + v[nU + nP:] @ (pc.C @ v[nU + nP:]))
        assert en(e) <= 1e-8 * en(xd), (prob.nx, k, en(e), en(xd))
    # the members of some set stopped at different iterations
    assert any(len(set(v)) > 1 for v in per_set.values() if len(v) > 1), per_set
    lbatch.close()
    plain.close()
    for s in solvers:
        s.close()
