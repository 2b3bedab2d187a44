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


def test_binding_checks_array_types_and_sizes_on_host():
    """The library takes bare pointers, so the binding refuses a tensor of the
    wrong element type or too few elements before anything is launched."""
    torch = pytest.importorskip("torch")
    from paper_2505_05587_gb300 import binding as B
    with pytest.raises(TypeError, match="image: dtype"):
        B._arr(torch.zeros(12, dtype=torch.float64), "image", B.F32, 12)
    with pytest.raises(TypeError, match="n_contrib: dtype"):
        B._arr(torch.zeros(4, dtype=torch.float32), "n_contrib", B.I32, 4)
    with pytest.raises(ValueError, match="S_accum: 11 elements, the call needs at least 12"):
        B._arr(torch.zeros(11), "S_accum", B.F32, 12)
    with pytest.raises(ValueError, match="CUDA device"):          # type and size fine: next, the device
        B._arr(torch.zeros(12), "S_accum", B.F32, 12)
    assert B._arr(None, "S_po", B.F32, 30) is None
    with pytest.raises(ValueError, match=r"\[H, W, 3\]"):
        B._image_hw(torch.zeros(4, 4))
    # the Gaussian arrays are checked against n and the SH degree
    g = B.GaussianTensors(torch.zeros(5, 3), torch.zeros(5, 3), torch.zeros(5, 4), torch.zeros(5),
                          torch.zeros(5, 9, 3), 3)
    with pytest.raises(ValueError, match="sh: 135 elements, the call needs at least 240"):
        g.ptrs()
    g.sh_degree = 4
    with pytest.raises(ValueError, match="sh_degree"):
        g.ptrs()
