"""The C-ABI library loads and exports every symbol include/mhfp.h declares
(no GPU needed: nothing is computed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mhfp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mhfp_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree():
    from paper_2002_09603_gb300 import EXPORTS
    assert sorted(EXPORTS) == _declared()


def test_library_exports_every_declared_symbol():
    from paper_2002_09603_gb300 import build
    try:
        path = build.build()
    except RuntimeError as e:  # no nvcc in this environment
        pytest.skip(str(e))
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_argument_validation_without_gpu():
    """mhfp_create rejects bad arguments on the host before touching a device."""
    from paper_2002_09603_gb300 import build
    import paper_2002_09603_gb300._lib as L
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    lib = L.load()
    h = ctypes.c_void_p()
    assert lib.mhfp_create(None, None, 1.0, None, None, ctypes.byref(h)) == 1
    assert lib.mhfp_status_string(5) == b"not converged"
    o = L.default_options()
    assert (o.restart, o.maxit, o.cheb_degree, o.coarse_max) == (50, 1000, 2, 125)


def _structs(prob):
    import numpy as np
    import paper_2002_09603_gb300._lib as L
    keep = {k: np.ascontiguousarray(getattr(prob, k)) for k in
            ("coords", "node_fix", "face_bc", "E", "nu", "biot", "Seps", "mu", "kappa")}
    mesh = L.Mesh(prob.nx, prob.ny, prob.nz, keep["coords"].ctypes.data, keep["node_fix"].ctypes.data,
                  keep["face_bc"].ctypes.data)
    mats = L.Materials(*(keep[k].ctypes.data for k in ("E", "nu", "biot", "Seps", "mu", "kappa")))
    return mesh, mats, keep


@pytest.mark.parametrize("field,value", [("nu", 0.5), ("E", -1.0), ("kappa", 0.0), ("mu", 0.0),
                                         ("Seps", -1e-9), ("nx", 0)])
def test_create_rejects_invalid_inputs_on_the_host(field, value):
    """Empty meshes and non-physical materials are rejected by mhfp_create
    before any device call (so this runs without a GPU)."""
    import mhfp_inputs as mi
    import paper_2002_09603_gb300._lib as L
    from paper_2002_09603_gb300 import build
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    prob = mi.random_small(2, 2, 2, seed=1)
    if field == "nx":
        prob.nx = value
    else:
        arr = getattr(prob, field).copy()
        arr.flat[3] = value
        setattr(prob, field, arr)
    mesh, mats, keep = _structs(prob)
    h = ctypes.c_void_p()
    trac = (ctypes.c_double * 3)(0.0, 0.0, -1.0)
    assert L.load().mhfp_create(ctypes.byref(mesh), ctypes.byref(mats), 0.1, trac, None, ctypes.byref(h)) == 1
    assert not h.value


def test_lockstep_batch_rejects_lane_counts_on_the_host():
    """mhfp_batch_create_lanes rejects a lane count outside 1..MHFP_MAX_LANES
    before it reads a handle (dummy pointers, no GPU)."""
    import paper_2002_09603_gb300._lib as L
    from paper_2002_09603_gb300 import build
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    src = open(os.path.join(ROOT, "include", "mhfp.h")).read()
    max_lanes = int(re.search(r"#define MHFP_MAX_LANES (\d+)", src).group(1))
    lib = L.load()
    dummy = (ctypes.c_void_p * 1)(ctypes.c_void_p(8))
    out = ctypes.c_void_p()
    for lanes in (0, -1, max_lanes + 1):
        assert lib.mhfp_batch_create_lanes(1, dummy, dummy, dummy, 1e-8, lanes, ctypes.byref(out)) == 1
        assert not out.value
    assert lib.mhfp_batch_create_lanes(1, dummy, dummy, dummy, 0.0, 2, ctypes.byref(out)) == 1
