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
