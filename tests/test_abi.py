"""C-ABI library: builds, loads, exports every declared symbol, and rejects
bad arguments on the host before any CUDA call (no GPU needed)."""
import ctypes as C
import re
import os

import numpy as np
import pytest

import paper_2605_28627_gb300 as dg
from workloads import box_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dgsem.h")).read()
    return sorted(set(re.findall(r"\b(dg_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert _declared() == sorted(dg.EXPORTS)


def test_library_exports_every_symbol():
    L = dg.load()
    for name in _declared():
        assert hasattr(L, name), name


def _init(mesh, N=3, **kw):
    L = dg.load()
    xgeo = np.ascontiguousarray(mesh.xgeo)
    nbr = np.ascontiguousarray(mesh.face_nbr, dtype=np.int32)
    m = dg.dg_mesh(xgeo.shape[0], xgeo.shape[-1] - 1, xgeo.ctypes.data_as(C.POINTER(C.c_double)),
                   nbr.ctypes.data_as(C.POINTER(C.c_int32)))
    prm = dict(N=N, gamma=1.4, R=1.0, Pr=0.72, mu=0.01, surf_flux=0, precision=0, source=0, mms_amp=0.1, p_ref=0.0, visc_law=0, T_ref=1.0, S_suth=0.0, nodes=0, rk_scheme=0)
    prm.update(kw)
    p = dg.dg_params(**prm)
    h = C.c_void_p()
    st = L.dg_init(C.byref(m), C.byref(p), 0, C.byref(h))
    return st, h, L.dg_last_error(None).decode()


def test_init_rejects_bad_arguments_on_host():
    m = box_mesh(2, 1, rotate_seed=1)
    st, h, msg = _init(m, N=0)
    assert st == dg.DG_EUNSUPPORTED and not h.value and "N" in msg
    st, h, msg = _init(m, N=10)
    assert st == dg.DG_EUNSUPPORTED and not h.value
    st, h, msg = _init(m, N=3, gamma=0.9)
    assert st == dg.DG_EINVAL and not h.value
    st, h, msg = _init(m, N=3, surf_flux=5)
    assert st == dg.DG_EINVAL
    bad = m.face_nbr.copy()
    bad[0, 0, 1] = (bad[0, 0, 1] + 1) % 6
    st, h, msg = _init(type(m)(**{**m.__dict__, "face_nbr": bad}))
    assert st == dg.DG_EMESH and "reciprocal" in msg
    bad = m.face_nbr.copy()
    bad[3, 2, 2] = 9
    st, h, msg = _init(type(m)(**{**m.__dict__, "face_nbr": bad}))
    assert st == dg.DG_EMESH and "range" in msg
    # an empty mesh (no elements) is an argument error, not a launch of empty grids
    empty = type(m)(**{**m.__dict__, "xgeo": m.xgeo[:0], "face_nbr": m.face_nbr[:0]})
    st, h, msg = _init(empty)
    assert st == dg.DG_EINVAL and not h.value
    L = dg.load()
    assert L.dg_init(None, None, 0, None) == dg.DG_EINVAL
    assert L.dg_state_len(None) == 0
    assert L.dg_time_derivative(None, None, None, 0.0, None) == dg.DG_EINVAL


def test_solver_refuses_to_run_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        dg.Solver(box_mesh(2, 1), 2)
