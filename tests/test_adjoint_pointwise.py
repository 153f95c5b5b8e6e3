"""Host check of the CUDA path's hand-written pointwise adjoints
(paper_2502_19342_gb300/csrc/physics_adj.cuh): the reverse-mode volume-node
and face-point functions against central finite differences of the forward
functions, for 1-3 species, inviscid and viscous (no GPU needed: the header
compiles for the host)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_pointwise_adjoints_match_finite_differences(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "adjcheck")
    subprocess.run([gxx, "-std=c++17", "-O1", "-o", exe, os.path.join(HERE, "adjoint_pointwise_check.cpp")],
                   check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
