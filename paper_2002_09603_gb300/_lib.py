"""ctypes binding of libmhfp (argument marshalling only).

Every computation runs in the CUDA library; this module converts numpy
inputs into the C structs, passes torch CUDA tensors as device pointers and
turns status codes into exceptions.  There is no CPU fallback: if the
shared library is missing the import of a Solver fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmhfp.so")

MHFP_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "invalid mesh", 3: "out of memory", 4: "CUDA error",
          5: "not converged", 6: "non-finite value", 7: "Krylov breakdown", 8: "call out of order"}

# every symbol include/mhfp.h declares
EXPORTS = ["mhfp_default_options", "mhfp_create", "mhfp_assemble_condense", "mhfp_setup_precond",
           "mhfp_build_rhs", "mhfp_solve", "mhfp_apply_operator", "mhfp_apply_operator_ff", "mhfp_apply_operator_t", "mhfp_adjoint_solve",
           "mhfp_grad_logk", "mhfp_misfit", "mhfp_adjoint_rhs", "mhfp_apply_precond_t", "mhfp_apply_precond", "mhfp_vcycle",
           "mhfp_level_apply", "mhfp_hierarchy", "mhfp_get_scalings", "mhfp_sizes", "mhfp_timing",
           "mhfp_timing_read", "mhfp_solve_batch", "mhfp_residual_norm_noalloc", "mhfp_update_logk",
           "mhfp_batch_create", "mhfp_batch_create_lanes", "mhfp_batch_run", "mhfp_batch_destroy", "mhfp_launch_count", "mhfp_last_error", "mhfp_status_string", "mhfp_destroy"]


class MhfpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Mesh(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("coords", C.c_void_p),
                ("node_fix", C.c_void_p), ("face_bc", C.c_void_p)]


class Materials(C.Structure):
    _fields_ = [("E", C.c_void_p), ("nu", C.c_void_p), ("biot", C.c_void_p), ("Seps", C.c_void_p),
                ("mu", C.c_void_p), ("kappa", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("restart", C.c_int), ("maxit", C.c_int), ("cheb_degree", C.c_int),
                ("cheb_ratio", C.c_double), ("coarse_max", C.c_int), ("power_iters", C.c_int),
                ("precision", C.c_int), ("graphs", C.c_int), ("autotune", C.c_int),
                ("reorth", C.c_int), ("schedule", C.c_int), ("fine_blocks", C.c_int),
                ("near_kernel", C.c_int), ("formulation", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("restarts", C.c_int), ("converged", C.c_int),
                ("rel_residual", C.c_double), ("true_rel_residual", C.c_double), ("solve_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class HierInfo(C.Structure):
    _fields_ = [("levels", C.c_int), ("points", C.c_longlong * 8), ("block", C.c_int * 8),
                ("lmax", C.c_double * 8), ("schedule", C.c_int * 8), ("sweep_us", C.c_double * 8),
                ("cheb_degree", C.c_int)]


_lib = None


def load(path: str | None = None):
    """Load libmhfp.so (built in-tree by paper_2002_09603_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libmhfp.so not built ({p}); run paper_2002_09603_gb300.build.build()")
    lib = C.CDLL(p)
    vp, i, d, ll = C.c_void_p, C.c_int, C.c_double, C.c_longlong
    sig = {
        "mhfp_default_options": (None, [C.POINTER(Options)]),
        "mhfp_create": (i, [C.POINTER(Mesh), C.POINTER(Materials), d, C.POINTER(C.c_double), vp, C.POINTER(vp)]),
        "mhfp_assemble_condense": (i, [vp]),
        "mhfp_setup_precond": (i, [vp, C.POINTER(Options)]),
        "mhfp_build_rhs": (i, [vp, vp, d, vp]),
        "mhfp_solve": (i, [vp, vp, vp, d, C.POINTER(Stats)]),
        "mhfp_apply_operator": (i, [vp, vp, vp]),
        "mhfp_apply_operator_ff": (i, [vp, vp, vp]),
        "mhfp_apply_precond": (i, [vp, vp, vp]),
        "mhfp_apply_operator_t": (i, [vp, vp, vp]),
        "mhfp_adjoint_solve": (i, [vp, vp, vp, d, C.POINTER(Stats)]),
        "mhfp_grad_logk": (i, [vp, vp, vp, vp]),
        "mhfp_apply_precond_t": (i, [vp, vp, vp]),
        "mhfp_misfit": (i, [vp, vp, vp, vp, d, d, vp, vp]),
        "mhfp_adjoint_rhs": (i, [vp, vp, vp, vp]),
        "mhfp_vcycle": (i, [vp, i, vp, vp]),
        "mhfp_level_apply": (i, [vp, i, i, vp, vp]),
        "mhfp_hierarchy": (i, [vp, i, C.POINTER(HierInfo)]),
        "mhfp_get_scalings": (i, [vp, vp, vp]),
        "mhfp_sizes": (i, [vp, C.POINTER(ll), C.POINTER(ll), C.POINTER(ll)]),
        "mhfp_timing": (i, [vp, i]),
        "mhfp_timing_read": (i, [vp, i, C.POINTER(ll), C.POINTER(d), C.POINTER(d)]),
        "mhfp_residual_norm_noalloc": (i, [vp, vp, vp, vp]),
        "mhfp_update_logk": (i, [vp, vp]),
        "mhfp_batch_create": (i, [i, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), d, C.POINTER(vp)]),
        "mhfp_batch_create_lanes": (i, [i, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), d, i, C.POINTER(vp)]),
        "mhfp_batch_run": (i, [vp, vp, C.POINTER(Stats), C.POINTER(i)]),
        "mhfp_batch_destroy": (None, [vp]),
        "mhfp_solve_batch": (i, [i, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), d, C.POINTER(Stats),
                                 C.POINTER(i)]),
        "mhfp_launch_count": (ll, []),
        "mhfp_last_error": (C.c_char_p, [vp]),
        "mhfp_status_string": (C.c_char_p, [i]),
        "mhfp_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def launch_count() -> int:
    """Kernels launched by libmhfp so far in this process."""
    return int(load().mhfp_launch_count())


def default_options() -> Options:
    o = Options()
    load().mhfp_default_options(C.byref(o))
    return o


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def check_vec(t, n, device, name, at_least=False):
    """Reject a tensor the C ABI would read or write out of bounds: it must be
    a float64, contiguous torch tensor on ``device`` with exactly ``n``
    elements (at least ``n`` when ``at_least``).  Raises ValueError."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a torch tensor, got {type(t).__name__}")
    if t.dtype != torch.float64:
        raise ValueError(f"{name}: expected float64, got {t.dtype}")
    if t.device != device:
        raise ValueError(f"{name}: expected a tensor on {device}, got {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: tensor is not contiguous")
    if (t.numel() < n) if at_least else (t.numel() != n):
        raise ValueError(f"{name}: expected {'at least ' if at_least else ''}{n} elements, got {t.numel()}")
    return t


class Solver:
    """One stabilized hybridized poromechanics system on one GPU.

    ``prob`` is an ``mhfp_inputs.Problem``.  Device vectors are float64
    torch CUDA tensors in the layout [u | p | pi]."""

    def __init__(self, prob, stream=None, device=None):
        import torch
        self.torch = torch
        self.lib = load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        torch.cuda.set_device(self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._keep = dict(
            coords=np.ascontiguousarray(prob.coords, dtype=np.float64),
            node_fix=np.ascontiguousarray(prob.node_fix, dtype=np.uint8),
            face_bc=np.ascontiguousarray(prob.face_bc, dtype=np.uint8),
            E=np.ascontiguousarray(prob.E, dtype=np.float64),
            nu=np.ascontiguousarray(prob.nu, dtype=np.float64),
            biot=np.ascontiguousarray(prob.biot, dtype=np.float64),
            Seps=np.ascontiguousarray(prob.Seps, dtype=np.float64),
            mu=np.ascontiguousarray(prob.mu, dtype=np.float64),
            kappa=np.ascontiguousarray(prob.kappa, dtype=np.float64),
        )
        k = self._keep
        mesh = Mesh(prob.nx, prob.ny, prob.nz, k["coords"].ctypes.data, k["node_fix"].ctypes.data,
                    k["face_bc"].ctypes.data)
        mats = Materials(k["E"].ctypes.data, k["nu"].ctypes.data, k["biot"].ctypes.data,
                         k["Seps"].ctypes.data, k["mu"].ctypes.data, k["kappa"].ctypes.data)
        trac = (C.c_double * 3)(*[float(v) for v in prob.traction])
        h = C.c_void_p()
        st = self.lib.mhfp_create(C.byref(mesh), C.byref(mats), float(prob.dt), trac,
                                  C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != MHFP_OK:
            raise MhfpError(st, "mhfp_create failed")
        self.h = h
        nu_, np_, npi = C.c_longlong(), C.c_longlong(), C.c_longlong()
        self.lib.mhfp_sizes(h, C.byref(nu_), C.byref(np_), C.byref(npi))
        self.sizes = (nu_.value, np_.value, npi.value)
        self.dims = (int(prob.nx), int(prob.ny), int(prob.nz))
        self.n = sum(self.sizes)

    # ------------------------------------------------------------ helpers
    def _check(self, st):
        if st != MHFP_OK:
            raise MhfpError(st, self.lib.mhfp_last_error(self.h).decode())

    def empty(self, n=None):
        return self.torch.empty(self.n if n is None else n, dtype=self.torch.float64, device=self.device)

    def _v(self, t, name, n=None, optional=False, at_least=False):
        """Device pointer of a checked vector (length n, default the system size)."""
        if t is None and optional:
            return None
        check_vec(t, self.n if n is None else n, self.device, name, at_least)
        return _ptr(t)

    def level_size(self, which, level):
        h = self.hierarchy(which)
        if not 0 <= level < h["levels"]:
            raise ValueError(f"level {level} out of range (hierarchy has {h['levels']})")
        return h["points"][level] * h["block"][level]

    # ------------------------------------------------------------ C ABI
    def assemble_condense(self):
        self._check(self.lib.mhfp_assemble_condense(self.h))

    def setup_precond(self, options: Options | None = None):
        self._check(self.lib.mhfp_setup_precond(self.h, None if options is None else C.byref(options)))
        self.formulation = 0 if options is None else int(options.formulation)

    def build_rhs(self, x_prev=None, load_scale=1.0, out=None):
        out = self.empty() if out is None else out
        self._check(self.lib.mhfp_build_rhs(self.h, self._v(x_prev, "x_prev", optional=True), float(load_scale),
                                            self._v(out, "out")))
        return out

    def solve(self, rhs, tol=1e-8, out=None, raise_not_converged=True):
        out = self.empty() if out is None else out
        st = Stats()
        code = self.lib.mhfp_solve(self.h, self._v(rhs, "rhs"), self._v(out, "out"), float(tol), C.byref(st))
        if code != MHFP_OK and not (code == 5 and not raise_not_converged):
            self._check(code)
        return out, st.as_dict()

    def apply_operator(self, x, out=None):
        out = self.empty() if out is None else out
        self._check(self.lib.mhfp_apply_operator(self.h, self._v(x, "x"), self._v(out, "out")))
        return out

    def apply_operator_ff(self, x, out=None):
        """y = A_H x as the mixed-precision Arnoldi step forms it: u rows in
        float-float arithmetic from x rounded to FP32 (mhfp_apply_operator_ff)."""
        out = self.empty() if out is None else out
        self._check(self.lib.mhfp_apply_operator_ff(self.h, self._v(x, "x"), self._v(out, "out")))
        return out

    def apply_operator_t(self, x, out=None):
        out = self.empty() if out is None else out
        self._check(self.lib.mhfp_apply_operator_t(self.h, self._v(x, "x"), self._v(out, "out")))
        return out

    def adjoint_solve(self, g, tol=1e-8, out=None, raise_not_converged=True):
        out = self.empty() if out is None else out
        st = Stats()
        code = self.lib.mhfp_adjoint_solve(self.h, self._v(g, "g"), self._v(out, "out"), float(tol), C.byref(st))
        if code != MHFP_OK and not (code == 5 and not raise_not_converged):
            self._check(code)
        return out, st.as_dict()

    def grad_logk(self, lam, x, grad):
        """grad -= lambda^T (dA/d ln kappa_T) x, per cell (accumulates)."""
        self._check(self.lib.mhfp_grad_logk(self.h, self._v(lam, "lam"), self._v(x, "x"),
                                            self._v(grad, "grad", n=self.sizes[1])))
        return grad

    def misfit(self, x, uz_target, p_target, inv_su2, inv_sp2, J, g):
        """J += step misfit (device scalar), g = its gradient."""
        ntop = self.uz_target_size()
        self._check(self.lib.mhfp_misfit(self.h, self._v(x, "x"), self._v(uz_target, "uz_target", n=ntop),
                                         self._v(p_target, "p_target", n=self.sizes[1]), float(inv_su2),
                                         float(inv_sp2), self._v(J, "J", n=1), self._v(g, "g")))
        return J, g

    def adjoint_rhs(self, g, lam_next, out=None):
        out = self.empty() if out is None else out
        self._check(self.lib.mhfp_adjoint_rhs(self.h, self._v(g, "g"), self._v(lam_next, "lam_next", optional=True),
                                              self._v(out, "out")))
        return out

    def apply_precond_t(self, v, out=None):
        out = self.empty() if out is None else out
        self._check(self.lib.mhfp_apply_precond_t(self.h, self._v(v, "v"), self._v(out, "out")))
        return out

    def apply_precond(self, v, out=None):
        out = self.empty() if out is None else out
        self._check(self.lib.mhfp_apply_precond(self.h, self._v(v, "v"), self._v(out, "out")))
        return out

    def vcycle(self, which, b, out=None):
        # which = 1: the interface-pressure hierarchy (n_pi), or C~_p's (n_p)
        # with the mixed formulation
        mixed = getattr(self, "formulation", 0) == 1
        n = self.sizes[0] if int(which) == 0 else self.sizes[1 if mixed else 2]
        out = self.empty(n) if out is None else out
        self._check(self.lib.mhfp_vcycle(self.h, int(which), self._v(b, "b", n=n), self._v(out, "out", n=n)))
        return out

    def level_apply(self, which, level, x, out=None):
        n = self.level_size(int(which), int(level))
        out = self.empty(n) if out is None else out
        self._check(self.lib.mhfp_level_apply(self.h, int(which), int(level), self._v(x, "x", n=n),
                                              self._v(out, "out", n=n)))
        return out

    def hierarchy(self, which):
        info = HierInfo()
        self._check(self.lib.mhfp_hierarchy(self.h, int(which), C.byref(info)))
        L = info.levels
        return dict(levels=L, points=list(info.points[:L]), block=list(info.block[:L]), lmax=list(info.lmax[:L]),
                    schedule=list(info.schedule[:L]), sweep_us=list(info.sweep_us[:L]),
                    cheb_degree=info.cheb_degree)

    def uz_target_size(self):
        """Top-plane node count (nx+1)(ny+1), the length of a u_z target."""
        return (self.dims[0] + 1) * (self.dims[1] + 1)

    def scalings(self):
        bt = self.empty(self.sizes[1])
        ds = self.empty()
        self._check(self.lib.mhfp_get_scalings(self.h, self._v(bt, "btilde", n=self.sizes[1]), self._v(ds, "ds")))
        return bt, ds

    def timing(self, enable: bool):
        self._check(self.lib.mhfp_timing(self.h, 1 if enable else 0))

    def timing_read(self, kernel_class: int):
        n, ms, b = C.c_longlong(), C.c_double(), C.c_double()
        self._check(self.lib.mhfp_timing_read(self.h, int(kernel_class), C.byref(n), C.byref(ms), C.byref(b)))
        return dict(launches=n.value, total_ms=ms.value, bytes_per_launch=b.value)

    def update_logk(self, logk):
        """New per-cell log-permeability (n_T float64 device values): the
        condensation, B~_p, C~_pi, D_s and the interface-pressure hierarchy
        are recomputed in place (mhfp_update_logk)."""
        self._check(self.lib.mhfp_update_logk(self.h, self._v(logk, "logk", n=self.sizes[1])))

    def residual_norm_noalloc(self, b, x, out=None):
        """(||D_s (b - A x)||, ||D_s b||) into a 2-element device tensor; the
        library allocates nothing for this call."""
        out = self.empty(2) if out is None else out
        self._check(self.lib.mhfp_residual_norm_noalloc(self.h, self._v(b, "b"), self._v(x, "x"),
                                                        self._v(out, "out", n=2, at_least=True)))
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.mhfp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(solvers, rhs, tol=1e-8, out=None):
    """Solve every solvers[i] with rhs[i] together (mhfp_solve_batch).
    Returns (xs, stats, statuses)."""
    import torch
    n = len(solvers)
    if len(rhs) != n or (out is not None and len(out) != n):
        raise ValueError("solve_batch: one right-hand side (and output) per solver")
    xs = out if out is not None else [s.empty() for s in solvers]
    for i, s in enumerate(solvers):
        check_vec(rhs[i], s.n, s.device, f"rhs[{i}]")
        check_vec(xs[i], s.n, s.device, f"out[{i}]")
    H = (C.c_void_p * n)(*[s.h.value for s in solvers])
    R = (C.c_void_p * n)(*[t.data_ptr() for t in rhs])
    X = (C.c_void_p * n)(*[t.data_ptr() for t in xs])
    st = (Stats * n)()
    codes = (C.c_int * n)()
    load().mhfp_solve_batch(n, H, R, X, float(tol), st, codes)
    return xs, [s.as_dict() for s in st], list(codes)


class Batch:
    """Many solves as one CUDA graph launch (mhfp_batch_*): entry i solves
    solvers[i] for rhs[i] into out[i]; entries of one solver run in order,
    different solvers concurrently.  The tensors are bound at creation.
    lanes > 1: a solver's entries in sets of up to `lanes` right-hand sides
    solved in lockstep (mhfp_batch_create_lanes)."""

    def __init__(self, solvers, rhs, out, tol=1e-8, lanes=1):
        n = len(solvers)
        if n == 0 or len(rhs) != n or len(out) != n:
            raise ValueError("Batch: one right-hand side and one output per entry")
        for i, s in enumerate(solvers):
            check_vec(rhs[i], s.n, s.device, f"rhs[{i}]")
            check_vec(out[i], s.n, s.device, f"out[{i}]")
        self.lib = load()
        self.solvers, self.rhs, self.out = list(solvers), list(rhs), list(out)
        H = (C.c_void_p * n)(*[s.h.value for s in solvers])
        R = (C.c_void_p * n)(*[t.data_ptr() for t in rhs])
        X = (C.c_void_p * n)(*[t.data_ptr() for t in out])
        b = C.c_void_p()
        if lanes == 1:
            code = self.lib.mhfp_batch_create(n, H, R, X, float(tol), C.byref(b))
        else:
            code = self.lib.mhfp_batch_create_lanes(n, H, R, X, float(tol), int(lanes), C.byref(b))
        if code != MHFP_OK:
            raise MhfpError(code, self.lib.mhfp_last_error(solvers[0].h).decode())
        self.b = b

    def run(self, stream=None):
        """One graph launch; returns (stats, statuses)."""
        n = len(self.solvers)
        st = (Stats * n)()
        codes = (C.c_int * n)()
        sp = C.c_void_p(stream.cuda_stream) if stream is not None else None
        code = self.lib.mhfp_batch_run(self.b, sp, st, codes)
        if code not in (MHFP_OK, 5, 6):  # a solve that did not converge is reported per entry
            raise MhfpError(code, self.lib.mhfp_last_error(self.solvers[0].h).decode())
        return [x.as_dict() for x in st], list(codes)

    def close(self):
        if getattr(self, "b", None):
            self.lib.mhfp_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def prepare(prob, options: Options | None = None, stream=None) -> Solver:
    """create -> assemble_condense -> setup_precond."""
    s = Solver(prob, stream=stream)
    s.assemble_condense()
    s.setup_precond(options)
    return s
