"""Host-side argument checks of the C ABI, called through ctypes with no GPU.

Each call below breaks exactly one rule of its entry point's contract and
must come back with SGS_ERR_INVALID_ARG (1) or SGS_ERR_WORKSPACE (2) before
anything is launched; the same call without that defect passes the checks and
fails only at the launch, with SGS_ERR_CUDA (4), as there is no device.  The array pointers are dummy addresses that the host
checks only compare; the module is skipped where a CUDA device is present so
that a check that stopped working could never launch on them."""
import ctypes as C

import pytest

import synth

torch = pytest.importorskip("torch")
if torch.cuda.is_available():
    pytest.skip("dummy-pointer host checks run only where no CUDA device exists", allow_module_level=True)

from paper_2505_05587_gb300 import binding as B  # noqa: E402
from paper_2505_05587_gb300 import build as bld  # noqa: E402

INVALID, WORKSPACE, NO_DEVICE = 1, 2, 4
DUMMY = 0x10000            # never dereferenced: the host checks fail first


@pytest.fixture(scope="module")
def lib():
    bld.build()
    return B.lib()          # the library with the binding's argument types


def _ptr(k=0):
    return C.c_void_p(DUMMY + 4096 * k)


def _gauss(n=10, sh_degree=0):
    return B.Gaussians(DUMMY, DUMMY + 4096, DUMMY + 8192, DUMMY + 12288, DUMMY + 16384, n, sh_degree)


def _mut(base=0x900000):
    return B.GaussiansMut(base, base + 4096, base + 8192, base + 12288, base + 16384)


def _view(tile=16):
    cam = synth.camera_identity(64, 48, 64.0)
    st = synth.Settings(tile_w=tile, tile_h=tile)
    return B.camera_c(cam), B.settings_c(st)


def _proj():
    return B.Proj(DUMMY, DUMMY, DUMMY, DUMMY, DUMMY, DUMMY)


def _bins(ranges=True):
    return B.Bins(DUMMY, None, DUMMY if ranges else None, DUMMY, 100, None)


def test_render_fwd_checks(lib):
    cam, st = _view()
    p, b = _proj(), _bins()
    ok = (C.byref(p), C.byref(b), C.byref(cam), C.byref(st), _ptr(1), _ptr(2), _ptr(3), None)
    assert lib.sgs_render_fwd(*ok) == NO_DEVICE
    nr = _bins(ranges=False)
    assert lib.sgs_render_fwd(ok[0], C.byref(nr), *ok[2:]) == INVALID          # no tile ranges
    wb = _bins()
    wb.walk, wb.walk_count = DUMMY + 40960, DUMMY + 45056                       # walk lists: both given
    assert lib.sgs_render_fwd(ok[0], C.byref(wb), *ok[2:]) == NO_DEVICE
    wb.walk_count = None                                                        # one without the other
    assert lib.sgs_render_fwd(ok[0], C.byref(wb), *ok[2:]) == INVALID
    assert lib.sgs_render_fwd(*ok[:4], None, *ok[5:]) == INVALID                # no image
    cam12, st12 = _view(tile=12)
    assert lib.sgs_render_fwd(ok[0], ok[1], C.byref(cam12), C.byref(st12), *ok[4:]) == INVALID   # tile 12x12
    bad_cam, _ = _view()
    bad_cam.fx = float("nan")
    assert lib.sgs_render_fwd(ok[0], ok[1], C.byref(bad_cam), *ok[3:]) == INVALID
    assert lib.sgs_render_fwd_l1(*ok[:4], _ptr(4), 0, _ptr(1), _ptr(2), _ptr(3), _ptr(5), _ptr(6),
                                 None) == INVALID                               # n_views < 1
    assert lib.sgs_render_stats(*ok[:4], None, None, None) == INVALID           # no counts
    assert lib.sgs_render_stats(*ok[:4], _ptr(9), None, None) == NO_DEVICE
    assert lib.sgs_render_stats(*ok[:4], _ptr(9), _ptr(10), None) == NO_DEVICE    # with per-block counts


def test_loss_checks(lib):
    assert lib.sgs_l1_loss_grad(_ptr(1), _ptr(2), 48, 64, 1, _ptr(3), _ptr(4), None) == NO_DEVICE
    assert lib.sgs_l1_loss_grad(_ptr(1), _ptr(2), 0, 64, 1, _ptr(3), _ptr(4), None) == INVALID
    assert lib.sgs_l1_loss_grad(_ptr(1), None, 48, 64, 1, _ptr(3), _ptr(4), None) == INVALID
    sz = C.c_size_t()
    assert lib.sgs_ssim_l1_workspace_size(48, 64, C.byref(sz)) == 0 and sz.value >= 9 * 48 * 64 * 4
    args = [_ptr(1), _ptr(2), 48, 64, 1, 1.5, _ptr(3), _ptr(4), _ptr(5), sz.value, None]
    assert lib.sgs_ssim_l1_loss_grad(*args) == INVALID                          # lambda outside [0, 1]
    args[5] = 0.2
    assert lib.sgs_ssim_l1_loss_grad(*args) == NO_DEVICE
    args[9] = sz.value - 1
    assert lib.sgs_ssim_l1_loss_grad(*args) == WORKSPACE


def test_backward_checks(lib):
    cam, st = _view()
    g, p, b = _gauss(), _proj(), _bins()
    grads = B.Grads(DUMMY, DUMMY, DUMMY, DUMMY, DUMMY)
    need = C.c_size_t()
    assert lib.sgs_render_bwd_workspace_size(10, C.byref(need)) == 0
    base = [C.byref(g), C.byref(p), C.byref(b), C.byref(cam), C.byref(st), _ptr(1), _ptr(2), _ptr(3),
            C.byref(grads), 0, _ptr(4), None, None, _ptr(7), need.value, None]
    assert lib.sgs_render_bwd_with_splitting(*base) == NO_DEVICE
    wb = _bins()
    wb.walk = DUMMY + 40960                                                     # walk without its counts
    a = list(base)
    a[2] = C.byref(wb)
    assert lib.sgs_render_bwd_with_splitting(*a) == INVALID
    wb.walk_count = DUMMY + 45056
    assert lib.sgs_render_bwd_with_splitting(*a) == NO_DEVICE
    for flags in (1, 2, 3):                                                     # accumulate grads, reset S, both
        a = list(base)
        a[9] = flags
        assert lib.sgs_render_bwd_with_splitting(*a) == NO_DEVICE
    for flags in (4, -1):                                                       # undefined flag bits
        a = list(base)
        a[9] = flags
        assert lib.sgs_render_bwd_with_splitting(*a) == INVALID
    a = list(base)
    a[12] = _ptr(6)                                                             # S_ls without S_po
    assert lib.sgs_render_bwd_with_splitting(*a) == INVALID
    a = list(base)
    a[10] = None                                                                # no S_accum, n > 0
    assert lib.sgs_render_bwd_with_splitting(*a) == INVALID
    a = list(base)
    a[14] = need.value - 1
    assert lib.sgs_render_bwd_with_splitting(*a) == WORKSPACE
    g3 = _gauss(sh_degree=4)
    a = list(base)
    a[0] = C.byref(g3)
    assert lib.sgs_render_bwd_with_splitting(*a) == INVALID


def test_densify_checks(lib):
    n = 10
    g = _gauss(n)
    need = C.c_size_t()
    assert lib.sgs_densify_split_workspace_size(n, C.byref(need)) == 0
    out = _mut()

    def call(**kw):
        a = dict(in_=C.byref(g), S=_ptr(1), S_po=None, S_ls=None, inv_T=1.0, eps=0.0, step=1.0, gn=None, eps_g=0.0,
                 budget=0, out=C.byref(out), cap=2 * n, d_n=_ptr(2), parent=None, lam=None, v=None, ws=_ptr(3),
                 ws_bytes=need.value, stream=None)
        a.update(kw)
        return lib.sgs_densify_split(*a.values())

    assert call() == NO_DEVICE
    assert call(cap=n - 1) == INVALID                                           # capacity below n
    assert call(inv_T=float("inf")) == INVALID
    assert call(S_ls=_ptr(5)) == INVALID                                        # S_ls without S_po
    alias = B.GaussiansMut(g.means, DUMMY + 0x100000, DUMMY + 0x200000, DUMMY + 0x300000, DUMMY + 0x400000)
    assert call(out=C.byref(alias)) == INVALID                                  # out aliases in
    assert call(d_n=None) == INVALID
    assert call(ws_bytes=need.value - 1) == WORKSPACE
    big = _gauss(1_000_001)                                                     # beyond the fixed scratch
    assert lib.sgs_densify_split_noalloc(C.byref(big), _ptr(1), None, None, 1.0, 0.0, 1.0, None, 0.0, 0,
                                         C.byref(out), 2_000_002, _ptr(2), None, None, None, None) == INVALID
    # the largest allowed n passes every size check (its workspace fits the
    # fixed array) and fails only for want of a device
    top = _gauss(1_000_000)
    assert lib.sgs_densify_split_noalloc(C.byref(top), _ptr(1), None, None, 1.0, 0.0, 1.0, None, 0.0, 0,
                                         C.byref(out), 2_000_000, _ptr(2), None, None, None, None) == NO_DEVICE


def test_clear_checks(lib):
    assert lib.sgs_clear(None, 0, None) == 0                                   # nothing to clear
    assert lib.sgs_clear(None, 16, None) == INVALID
    assert lib.sgs_clear(_ptr(1), 16, None) == NO_DEVICE


def test_adam_and_probe_checks(lib):
    args = [_ptr(1), _ptr(2), _ptr(3), _ptr(4), 100, 1e-3, 0.9, 0.999, 1e-8, 1, None, None]
    assert lib.sgs_adam_step(*args) == NO_DEVICE
    for k, bad in ((9, 0), (6, 1.0), (8, 0.0), (5, -1.0), (4, -1)):
        a = list(args)
        a[k] = bad
        assert lib.sgs_adam_step(*a) == INVALID, (k, bad)
    a = list(args)
    a[1] = None                                                                 # no grad with count > 0
    assert lib.sgs_adam_step(*a) == INVALID
    a = list(args)
    a[9] = _ptr(5)
    assert lib.sgs_adam_step_dev(*a) == NO_DEVICE
    a[9] = None                                                                 # no device step count
    assert lib.sgs_adam_step_dev(*a) == INVALID
    assert lib.sgs_fma_probe(_ptr(1), 4, 10, None) == NO_DEVICE
    assert lib.sgs_fma_probe(_ptr(1), 0, 10, None) == INVALID


def test_batched_checks(lib):
    cam, st = _view()
    cams = (B.Camera * 17)(*([cam] * 17))
    g = _gauss()
    grads = B.Grads(DUMMY, DUMMY, DUMMY, DUMMY, DUMMY)
    sz = C.c_size_t()
    assert lib.sgs_render_views_workspace_size(10, cams, 17, C.byref(st), 1000, C.byref(sz)) == INVALID
    assert lib.sgs_render_views_workspace_size(10, cams, 2, C.byref(st), 1000, C.byref(sz)) == 0
    base = [C.byref(g), cams, 2, C.byref(st), 128, _ptr(1), _ptr(2), _ptr(3), C.byref(grads), 0, _ptr(4), None,
            _ptr(5), 1000, _ptr(6), sz.value, None]
    assert lib.sgs_render_views_with_splitting(*base) == NO_DEVICE
    a = list(base)
    a[9] = 8                                                                    # undefined flag bit
    assert lib.sgs_render_views_with_splitting(*a) == INVALID
    a = list(base)
    a[4] = 100                                                                  # batch not 64/128/256
    assert lib.sgs_render_views_with_splitting(*a) == INVALID
    a = list(base)
    a[15] = sz.value - 1
    assert lib.sgs_render_views_with_splitting(*a) == WORKSPACE
    # the binning inside the workspace: pointers into ws, no launch, no device needed
    b = B.Bins()
    assert lib.sgs_render_views_bins(10, cams, 2, C.byref(st), 1000, _ptr(6), sz.value - 1, C.byref(b)) == WORKSPACE
    assert lib.sgs_render_views_bins(10, cams, 2, C.byref(st), 1000, _ptr(6), sz.value, None) == INVALID
    assert lib.sgs_render_views_bins(10, cams, 2, C.byref(st), 1000, _ptr(6), sz.value, C.byref(b)) == 0
    lo, hi = DUMMY + 4096 * 6, DUMMY + 4096 * 6 + sz.value
    for p in (b.gids, b.ranges, b.order):
        assert lo <= p < hi
    assert b.capacity == 1000 and not b.keys and not b.count and not b.walk
    scenes = (B.Gaussians * 2)(_gauss(10, 0), _gauss(10, 1))                    # SH degrees differ
    assert lib.sgs_render_batch_workspace_size(scenes, cams, 2, C.byref(st), 1000, C.byref(sz)) == INVALID
