"""mhfp_residual_norm_noalloc: the residual check for callers that cannot
allocate device memory at the point of the call (hosts whose device memory
belongs to their own pool allocator, loops that must not allocate once
running).  It must agree with the allocating path -- mhfp_solve's reported
true residual and D_s (b - A x) formed from mhfp_apply_operator -- on two
calls in a row, since every call reuses the same static scratch array.

This file sorts last so that a run stopping at the first failure has run
every other test first; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import mhfp_inputs as mi

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_residual_norm_without_allocation_matches_allocating_path():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2002_09603_gb300 import prepare

    s = prepare(mi.random_small(6, 5, 4, seed=7, jitter=0.1))
    b = s.build_rhs()
    x, st = s.solve(b, tol=1e-6)
    _, ds = s.scalings()
    rng = np.random.default_rng(11)
    x2 = torch.from_numpy(rng.standard_normal(s.n)).cuda()
    for xx, expect_rel in ((x, st["true_rel_residual"]), (x2, None), (x, st["true_rel_residual"])):
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        s.residual_norm_noalloc(b, xx, out)
        torch.cuda.synchronize()
        rn, bn = out.cpu().numpy()
        ax = s.apply_operator(xx)
        ref_r = torch.linalg.vector_norm(ds * (b - ax)).item()
        ref_b = torch.linalg.vector_norm(ds * b).item()
        ref_ax = torch.linalg.vector_norm(ds * ax).item()
        # the two paths sum A x in different orders, so their rounding is
        # relative to the size of the terms, ||D_s b|| + ||D_s A x||, not to
        # the residual (small after a solve, where b - A x cancels)
        assert abs(bn - ref_b) <= 1e-12 * ref_b, (bn, ref_b)
        assert abs(rn - ref_r) <= 1e-12 * (ref_b + ref_ax), (rn, ref_r)
        if expect_rel is not None:
            assert abs(rn / bn - expect_rel) <= 1e-12, (rn / bn, expect_rel)
    s.close()
