"""Host test of the resident engine's point order (csrc/resident_order.h).

The header is plain C++ shared by host and device code; this compiles a small
checker against it with the host compiler and runs it: the numbering must be a
bijection onto the tile plus its ring, and the point sets that each step of a
block of iterations updates must be prefixes of the numbering."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1712_10279_gb300", "csrc")


def test_resident_point_order():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "order_check")
        subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "native", "resident_order_check.cpp"),
                        "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok ")
