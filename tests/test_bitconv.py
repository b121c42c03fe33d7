"""Host checks of the stacking kernel's number helpers, compiled for the host
from the same headers as the kernel:

* the integer-pipe conversions (FP64 -> FP32 truncated and rounded, FP32 ->
  FP64) against the host's conversions on special values, every neighbour
  of the integers and half-integers of the image range, FP32 rounding ties
  and random bit patterns (tests/native/check_bitconv.cpp);
* the double-float helpers of the TAN projection (FP64 split, dot product,
  quotient, floor) against long double, and the whole projection at 0.2
  arcsec pixels to 5e-8 px (tests/native/check_dfloat.cpp)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(tmp_path, name):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / name
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2503_08854_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", name + ".cpp"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout[-2000:]
    return out.stdout


def test_integer_pipe_conversions(tmp_path):
    out = _run(tmp_path, "check_bitconv")
    assert out.startswith("ok ") and int(out.split()[1]) > 10_000_000


def test_double_float_projection(tmp_path):
    out = _run(tmp_path, "check_dfloat")
    assert out.strip().endswith("ok"), out
