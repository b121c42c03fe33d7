"""The integer-pipe conversions of the stacking kernel (FP64 -> FP32
truncated and rounded, FP32 -> FP64, floor to int) compiled for the host and
checked against the host's conversions and std::floor: special values, every
neighbour of the integers and half-integers of the image range, FP32 rounding
ties and random bit patterns (tests/native/check_bitconv.cpp)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_integer_pipe_conversions(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "check_bitconv"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2503_08854_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "check_bitconv.cpp"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout[-2000:]
    assert out.stdout.startswith("ok ") and int(out.stdout.split()[1]) > 10_000_000
