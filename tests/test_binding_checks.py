"""The binding rejects tensors that the C ABI would read or write out of
bounds (wrong dtype, device, layout or length) before it calls the library.
Runs on the CPU: the library is replaced by a recorder, so nothing launches."""
import pytest

torch = pytest.importorskip("torch")

from paper_2002_09603_gb300 import _lib  # noqa: E402


class _Recorder:
    """Stands in for libmhfp: records every call and returns MHFP_OK."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def f(*args):
            self.calls.append(name)
            return 0
        return f


def _solver(n_u=6, n_p=2, n_pi=5):
    s = _lib.Solver.__new__(_lib.Solver)
    s.torch = torch
    s.lib = _Recorder()
    s.h = None
    s.device = torch.device("cpu")
    s.sizes = (n_u, n_p, n_pi)
    s.n = sum(s.sizes)
    s.dims = (1, 1, 1)
    return s


def _good(n):
    return torch.zeros(n, dtype=torch.float64)


def test_check_vec_accepts_and_rejects():
    dev = torch.device("cpu")
    assert _lib.check_vec(_good(7), 7, dev, "v") is not None
    assert _lib.check_vec(_good(9), 7, dev, "v", at_least=True) is not None
    bad = [
        (torch.zeros(7, dtype=torch.float32), "float64"),
        (torch.zeros(14, dtype=torch.float64)[::2], "contiguous"),
        (_good(6), "7 elements"),
        (_good(8), "7 elements"),
        ([0.0] * 7, "torch tensor"),
    ]
    for t, msg in bad:
        with pytest.raises(ValueError, match=msg):
            _lib.check_vec(t, 7, dev, "v")
    with pytest.raises(ValueError, match="at least 3"):
        _lib.check_vec(_good(2), 3, dev, "out", at_least=True)
    with pytest.raises(ValueError, match="expected a tensor on"):
        _lib.check_vec(_good(7), 7, torch.device("meta"), "v")


@pytest.mark.parametrize("call", ["apply_operator", "apply_operator_ff", "apply_operator_t", "apply_precond", "apply_precond_t"])
def test_operator_wrappers_validate_before_calling(call):
    s = _solver()
    getattr(s, call)(_good(s.n), out=_good(s.n))
    assert len(s.lib.calls) == 1
    for x, out in [(_good(s.n - 1), _good(s.n)), (_good(s.n), _good(s.n + 1)),
                   (_good(s.n).float(), _good(s.n)), (torch.zeros(2 * s.n, dtype=torch.float64)[::2], _good(s.n))]:
        with pytest.raises(ValueError):
            getattr(s, call)(x, out=out)
    assert len(s.lib.calls) == 1


def test_solve_rhs_noalloc_and_gradient_wrappers_validate():
    s = _solver()
    with pytest.raises(ValueError):
        s.solve(_good(s.n - 1), out=_good(s.n))
    with pytest.raises(ValueError):
        s.build_rhs(x_prev=_good(3), out=_good(s.n))
    s.build_rhs(x_prev=None, out=_good(s.n))
    with pytest.raises(ValueError, match="at least 2"):
        s.residual_norm_noalloc(_good(s.n), _good(s.n), out=_good(1))
    s.residual_norm_noalloc(_good(s.n), _good(s.n), out=_good(2))
    with pytest.raises(ValueError):
        s.grad_logk(_good(s.n), _good(s.n), _good(s.sizes[1] + 1))
    s.grad_logk(_good(s.n), _good(s.n), _good(s.sizes[1]))
    with pytest.raises(ValueError):
        s.misfit(_good(s.n), _good(3), _good(s.sizes[1]), 1.0, 1.0, _good(1), _good(s.n))
    s.misfit(_good(s.n), _good(4), _good(s.sizes[1]), 1.0, 1.0, _good(1), _good(s.n))
    with pytest.raises(ValueError):
        s.vcycle(0, _good(s.sizes[2]))
    assert s.lib.calls == ["mhfp_build_rhs", "mhfp_residual_norm_noalloc", "mhfp_grad_logk", "mhfp_misfit"]


def test_batch_wrapper_validates():
    s1, s2 = _solver(), _solver(3, 1, 2)
    with pytest.raises(ValueError, match="rhs\\[1\\]"):
        _lib.solve_batch([s1, s2], [_good(s1.n), _good(s1.n)], out=[_good(s1.n), _good(s2.n)])
    with pytest.raises(ValueError, match="one right-hand side"):
        _lib.solve_batch([s1, s2], [_good(s1.n)])
