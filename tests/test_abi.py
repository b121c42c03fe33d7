"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/ndt.h declares (no device calls: runs without a GPU)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ndt_\w+)\s*\(", src, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2503_08854_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ndt_create", "ndt_destroy", "ndt_load_exposures", "ndt_stack_orbits",
              "ndt_topk_candidates", "ndt_predict_positions", "ndt_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_uses_only_declared_symbols(lib):
    from paper_2503_08854_gb300 import ndt
    assert set(ndt.exported_symbols()) <= _declared()


def test_create_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2503_08854_gb300 import ndt
    with pytest.raises(ndt.NdtError):
        ndt.create(0)
