"""CPU checks of the C ABI library: it loads without a GPU and exports every
entry point include/rm.h declares; the binding's structs match the header."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(rm_[a-z_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = _declared()
    for want in ["rm_setup", "rm_apply", "rm_precondition", "rm_solve", "rm_ndofs",
                 "rm_destroy", "rm_last_error", "rm_default_options", "rm_stats"]:
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2211_14284_gb300 import rm
    lib = rm.load()
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) <= set(rm.EXPORTED)


def test_default_options_struct_layout():
    from paper_2211_14284_gb300 import rm
    o = rm.load().rm_default_options()
    assert o.rtol == 1e-8 and o.max_it == 500 and o.check_every == 1
    assert o.precision == rm.RM_FP64 and o.coarse == rm.RM_COARSE_P1 and o.profile == 0


def test_setup_without_gpu_fails_loudly():
    """No CPU fallback: without a usable CUDA device rm_setup returns an
    error (RM_ERR_CUDA or an argument error), never a result."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2211_14284_gb300.rm import RmError, Solver
    with pytest.raises(RmError):
        Solver(0, 2, 2)
