"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every function that include/steepgs.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(sgs_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("sgs_project", "sgs_bin_sort", "sgs_render_fwd", "sgs_render_bwd_with_splitting",
                     "sgs_densify_split", "sgs_l1_loss_grad"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2505_05587_gb300 import build as bld
    path = bld.build()
    lib = ctypes.CDLL(path)
    for name in _declared_functions():
        assert hasattr(lib, name), name
    lib.sgs_error_string.restype = ctypes.c_char_p
    assert lib.sgs_error_string(0) == b"ok"
    assert lib.sgs_version() >= 100


def test_host_side_argument_checks_without_gpu():
    """Calls that fail validation return before touching CUDA."""
    from paper_2505_05587_gb300 import build as bld
    lib = ctypes.CDLL(bld.build())
    assert lib.sgs_project(None, None, None, None, None) == 1
    sz = ctypes.c_size_t()
    assert lib.sgs_bin_sort_workspace_size(-1, 10, 4, ctypes.byref(sz)) == 1
    assert lib.sgs_bin_sort_workspace_size(100, 1000, 16, ctypes.byref(sz)) == 0 and sz.value > 0
    assert lib.sgs_densify_split_workspace_size(100, ctypes.byref(sz)) == 0 and sz.value > 0
    assert lib.sgs_render_bwd_workspace_size(100, ctypes.byref(sz)) == 0 and sz.value >= 100 * 64
