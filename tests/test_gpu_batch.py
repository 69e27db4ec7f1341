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
