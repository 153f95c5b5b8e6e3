"""The C-ABI library loads and exports every entry point include/dgfv.h declares
(no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dgfv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dgfv_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("dgfv_init_mesh", "dgfv_set_state", "dgfv_set_degrees", "dgfv_eval_rhs", "dgfv_rk_step",
                     "dgfv_adapt"):
        assert required in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_2502_19342_gb300 import build
    try:
        path = build.build()
    except RuntimeError as e:  # no CUDA toolkit on this host
        pytest.skip(str(e))
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2502_19342_gb300 import dgfv
    assert set(dgfv.SYMBOLS) == set(_declared())


def test_binding_refuses_to_run_without_the_library(monkeypatch, tmp_path):
    from paper_2502_19342_gb300 import dgfv
    monkeypatch.setattr(dgfv, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(dgfv, "_lib", None)
    with pytest.raises(RuntimeError):
        dgfv.lib()


def _lib_or_skip():
    from paper_2502_19342_gb300 import build, dgfv
    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    return dgfv, dgfv.lib()


def test_init_mesh_refuses_bad_meshes_before_touching_the_device():
    """The argument checks of dgfv_init_mesh that precede any CUDA call: a
    null pointer, no domains, an empty or inverted domain, degrees outside
    1..7, N_FV below N_max + 1 or above 9, more than three species, and an FV
    element whose sub-cell data would not fit one CTA's shared memory."""
    dgfv, L = _lib_or_skip()
    import ctypes as C
    import numpy as np

    def init(n_domains=1, dims=(2, 2, 2), lo=(0, 0, 0), hi=(1, 1, 1), N_min=1, N_max=4, N_fv=5, nk=2, null=False):
        d = np.ascontiguousarray(dims, np.int32)
        a = np.ascontiguousarray(lo, np.float64)
        b = np.ascontiguousarray(hi, np.float64)
        mesh = dgfv.MeshDesc(n_domains, d.ctypes.data_as(C.POINTER(C.c_int32)),
                             a.ctypes.data_as(C.POINTER(C.c_double)), b.ctypes.data_as(C.POINTER(C.c_double)),
                             N_min, N_max, N_fv, 0)
        ph = dgfv.Phys()
        ph.n_species = nk
        for k in range(3):
            ph.gamma[k], ph.Rgas[k], ph.Pr[k] = 1.4, 1.0, 0.72
        op = dgfv.Opts(0, 0.5, 0.5, 1.0, 1.6, 3.0, 7.0, 0, 0, 0, 0, 0, 1e-10)
        h = C.c_void_p()
        rc = L.dgfv_init_mesh(C.byref(h), None if null else C.byref(mesh), C.byref(ph), C.byref(op))
        return rc, h.value

    ERR_ARG = -1
    for kw in (dict(null=True), dict(n_domains=0), dict(dims=(0, 2, 2)), dict(hi=(1, 0, 1)), dict(N_min=0),
               dict(N_max=8, N_fv=9), dict(N_min=5, N_max=4), dict(N_fv=4), dict(N_fv=10), dict(nk=4), dict(nk=0),
               dict(N_max=7, N_fv=9, nk=3)):
        rc, h = init(**kw)
        assert rc == ERR_ARG and not h, kw


def test_calls_on_a_null_context_and_status_strings():
    """Every status has its own message; calls on a null context are refused
    with DGFV_ERR_ARG, and destroying a null context is a no-op."""
    dgfv, L = _lib_or_skip()
    import ctypes as C
    L.dgfv_status_string.restype = C.c_char_p
    msgs = [L.dgfv_status_string(s) for s in range(0, -8, -1)]
    assert all(msgs) and len(set(msgs)) == 8
    assert L.dgfv_status_string(-99) == b"unknown status"
    L.dgfv_last_error.restype = C.c_char_p
    assert L.dgfv_last_error(None) == b"null context"
    ERR_ARG = -1
    assert L.dgfv_eval_rhs(None, None, None, None) == ERR_ARG
    assert L.dgfv_set_state(None, None, 0, None) == ERR_ARG
    assert L.dgfv_rhs_vjp(None, None, None, None, None) == ERR_ARG
    assert L.dgfv_rk_step(None, -1.0, None, None) == ERR_ARG
    assert L.dgfv_rk_step_vjp(None, None, 1e-3, None, None, None) == ERR_ARG
    L.dgfv_destroy(None)
