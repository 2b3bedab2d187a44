"""Thin Python binding of libsteepgs (include/steepgs.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  PyTorch provides device memory and the stream.  There is no CPU
fallback: if the library is missing, importing this module raises.

Functions keep the C names without the ``sgs_`` prefix: project, bin_sort,
render_fwd, l1_loss_grad, render_bwd_with_splitting, densify_split, and the
workspace-size queries.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsteepgs.so")

SGS_OK = 0
ERRORS = {1: "invalid argument", 2: "workspace too small", 3: "capacity exceeded", 4: "CUDA error",
          5: "timeout", 6: "unsupported"}


class SteepGSError(RuntimeError):
    def __init__(self, fn: str, status: int, cuda: int = 0):
        msg = f"{fn}: {ERRORS.get(status, 'unknown')} (status {status})"
        if status == 4:
            msg += f", cudaError {cuda}"
        super().__init__(msg)
        self.status = status


# --------------------------------------------------------------------------
# ctypes mirrors of the C structs
# --------------------------------------------------------------------------
class Gaussians(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int32),
                ("sh_degree", C.c_int32)]


class GaussiansMut(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p)]


class Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("near_z", C.c_float)]


class Settings(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("alpha_min", C.c_float),
                ("alpha_max", C.c_float), ("T_min", C.c_float), ("radius_sigma", C.c_float),
                ("dilation", C.c_float), ("fov_clamp", C.c_float), ("bg", C.c_float * 3)]


class Proj(C.Structure):
    _fields_ = [("xy", C.c_void_p), ("conic_opac", C.c_void_p), ("rgb", C.c_void_p),
                ("depth", C.c_void_p), ("rect", C.c_void_p), ("tiles_touched", C.c_void_p)]


class Bins(C.Structure):
    _fields_ = [("gids", C.c_void_p), ("keys", C.c_void_p), ("ranges", C.c_void_p),
                ("count", C.c_void_p), ("capacity", C.c_int64), ("order", C.c_void_p),
                ("walk", C.c_void_p), ("walk_count", C.c_void_p)]


class Grads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p)]


_lib = None


def lib():
    """Loads libsteepgs.so; raises (no fallback) when it is not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libsteepgs.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        P, I32, I64, F, SZ = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_size_t
        L.sgs_error_string.restype = C.c_char_p
        L.sgs_error_string.argtypes = [C.c_int]
        L.sgs_get_last_cuda_error.restype = C.c_int
        L.sgs_version.restype = C.c_int
        L.sgs_kernel_launches.restype = C.c_uint64
        L.sgs_project.argtypes = [P, P, P, P, P]
        L.sgs_bin_sort_workspace_size.argtypes = [I32, I64, I32, C.POINTER(SZ)]
        L.sgs_bin_sort.argtypes = [P, I32, P, P, P, P, SZ, P]
        L.sgs_render_fwd.argtypes = [P, P, P, P, P, P, P, P]
        L.sgs_render_fwd_l1.argtypes = [P, P, P, P, P, I32, P, P, P, P, P, P]
        L.sgs_l1_loss_grad.argtypes = [P, P, I32, I32, I32, P, P, P]
        L.sgs_render_stats.argtypes = [P, P, P, P, P, P, P]
        L.sgs_render_bwd_workspace_size.argtypes = [I32, C.POINTER(SZ)]
        L.sgs_render_bwd_with_splitting.argtypes = [P, P, P, P, P, P, P, P, P, I32, P, P, P, P, SZ, P]
        L.sgs_densify_split_workspace_size.argtypes = [I32, C.POINTER(SZ)]
        L.sgs_densify_split.argtypes = [P, P, P, P, F, F, F, P, F, I64, P, I64, P, P, P, P, P, SZ, P]
        L.sgs_render_views_workspace_size.argtypes = [I32, P, I32, P, I64, C.POINTER(SZ)]
        L.sgs_render_views_workspace_size.restype = C.c_int
        L.sgs_render_views_with_splitting.argtypes = [P, P, I32, P, I32, P, P, P, P, I32, P, P, P, I64, P, SZ, P]
        L.sgs_render_views_with_splitting.restype = C.c_int
        L.sgs_render_batch_workspace_size.argtypes = [P, P, I32, P, I64, C.POINTER(SZ)]
        L.sgs_render_batch_workspace_size.restype = C.c_int
        L.sgs_render_batch_fwd.argtypes = [P, P, I32, P, I32, P, P, I64, P, SZ, P]
        L.sgs_render_batch_fwd.restype = C.c_int
        L.sgs_adam_step.argtypes = [P, P, P, P, I64, F, F, F, F, I32, P, P]
        L.sgs_adam_step_dev.argtypes = [P, P, P, P, I64, F, F, F, F, P, P, P]
        L.sgs_adam_step.restype = C.c_int
        L.sgs_ssim_l1_workspace_size.argtypes = [I32, I32, C.POINTER(SZ)]
        L.sgs_ssim_l1_workspace_size.restype = C.c_int
        L.sgs_ssim_l1_loss_grad.argtypes = [P, P, I32, I32, I32, F, P, P, P, SZ, P]
        L.sgs_ssim_l1_loss_grad.restype = C.c_int
        L.sgs_fma_probe.argtypes = [P, I32, I32, P]
        L.sgs_fma_probe.restype = C.c_int
        L.sgs_densify_split_noalloc.argtypes = [P, P, P, P, F, F, F, P, F, I64, P, I64, P, P, P, P, P]
        L.sgs_render_views_bins.argtypes = [I32, P, I32, P, I64, P, SZ, P]
        L.sgs_render_views_bins.restype = C.c_int
        L.sgs_clear.argtypes = [P, SZ, P]
        L.sgs_clear.restype = C.c_int
        for name in ("sgs_project", "sgs_bin_sort_workspace_size", "sgs_bin_sort", "sgs_render_fwd",
                     "sgs_l1_loss_grad", "sgs_render_stats", "sgs_render_bwd_workspace_size", "sgs_render_bwd_with_splitting",
                     "sgs_densify_split_workspace_size", "sgs_densify_split", "sgs_densify_split_noalloc"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(fn: str, status: int):
    if status != SGS_OK:
        raise SteepGSError(fn, status, lib().sgs_get_last_cuda_error())


def _p(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


F32 = (torch.float32,)
I16 = (torch.int16,)
I32 = tuple(d for d in (torch.int32, getattr(torch, "uint32", None)) if d is not None)
I64 = tuple(d for d in (torch.int64, getattr(torch, "uint64", None)) if d is not None)


def _check_arr(t, name: str, dtypes, numel: int = 0):
    """Checks the element type of `t` (None passes) and that it holds at least
    `numel` elements.  The library receives bare pointers and cannot check the
    arrays behind them, so a tensor too small for the call is refused here,
    before anything is launched."""
    if t is None:
        return
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch.Tensor")
    if t.dtype not in dtypes:
        raise TypeError(f"{name}: dtype {t.dtype}, expected {' or '.join(str(d) for d in dtypes)}")
    if t.numel() < numel:
        raise ValueError(f"{name}: {t.numel()} elements, the call needs at least {numel}")


def _arr(t, name: str, dtypes, numel: int = 0):
    """Device pointer of `t` (None passes through) after _check_arr."""
    _check_arr(t, name, dtypes, numel)
    return _p(t)


def _pixels(cam) -> int:
    return int(cam.width) * int(cam.height)


def _stream(stream):
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


# --------------------------------------------------------------------------
# Tensor bundles
# --------------------------------------------------------------------------
@dataclass
class GaussianTensors:
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logit: torch.Tensor
    sh: torch.Tensor
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def ptrs(self, rows: int | None = None, what: str = "") -> tuple:
        """Device pointers of the five arrays, each checked to hold `rows`
        (default n) Gaussians of this SH degree."""
        r = self.n if rows is None else int(rows)
        if not 0 <= self.sh_degree <= 3:
            raise ValueError(f"sh_degree {self.sh_degree} outside 0..3")
        K = (self.sh_degree + 1) ** 2
        arrays = ((self.means, "means", 3 * r), (self.log_scales, "log_scales", 3 * r), (self.quats, "quats", 4 * r),
                  (self.opacity_logit, "opacity_logit", r), (self.sh, "sh", 3 * K * r))
        for t, name, k in arrays:
            _check_arr(t, what + name, F32, k)
        return tuple(_p(t) for t, _, _ in arrays)

    def c(self) -> Gaussians:
        return Gaussians(*self.ptrs(), self.n, self.sh_degree)

    def c_mut(self, rows: int | None = None) -> GaussiansMut:
        return GaussiansMut(*self.ptrs(rows, "out."))

    def grads_c(self, g: "GaussianTensors") -> "Grads":
        """These tensors as the gradient arrays of the Gaussians `g`."""
        if self.sh_degree != g.sh_degree:
            raise ValueError("gradients and Gaussians differ in SH degree")
        return Grads(*self.ptrs(g.n, "grads."))

    @staticmethod
    def empty(n: int, sh_degree: int, device="cuda") -> "GaussianTensors":
        K = (sh_degree + 1) ** 2
        f = dict(device=device, dtype=torch.float32)
        return GaussianTensors(torch.empty(n, 3, **f), torch.empty(n, 3, **f), torch.empty(n, 4, **f),
                               torch.empty(n, **f), torch.empty(n, K, 3, **f), sh_degree)

    @staticmethod
    def from_scene(scene, device="cuda") -> "GaussianTensors":
        f = dict(device=device, dtype=torch.float32)
        return GaussianTensors(torch.as_tensor(scene.means).to(**f).contiguous(),
                               torch.as_tensor(scene.log_scales).to(**f).contiguous(),
                               torch.as_tensor(scene.quats).to(**f).contiguous(),
                               torch.as_tensor(scene.opacity_logit).to(**f).contiguous(),
                               torch.as_tensor(scene.sh).to(**f).contiguous(), int(scene.sh_degree))

    def zeros_like(self) -> "GaussianTensors":
        return GaussianTensors(torch.zeros_like(self.means), torch.zeros_like(self.log_scales),
                               torch.zeros_like(self.quats), torch.zeros_like(self.opacity_logit),
                               torch.zeros_like(self.sh), self.sh_degree)

    def narrow(self, n: int) -> "GaussianTensors":
        return GaussianTensors(self.means[:n], self.log_scales[:n], self.quats[:n], self.opacity_logit[:n],
                               self.sh[:n], self.sh_degree)

    def tensors(self):
        return (self.means, self.log_scales, self.quats, self.opacity_logit, self.sh)


@dataclass
class ProjBuffers:
    xy: torch.Tensor           # [N,4] f32
    conic_opac: torch.Tensor   # [N,4] f32
    rgb: torch.Tensor          # [N,4] f32
    depth: torch.Tensor        # [N]   f32
    rect: torch.Tensor         # [N,4] i16
    tiles_touched: torch.Tensor  # [N] i32 (uint32 in C)

    @staticmethod
    def alloc(n: int, device="cuda") -> "ProjBuffers":
        f = dict(device=device, dtype=torch.float32)
        return ProjBuffers(torch.empty(n, 4, **f), torch.empty(n, 4, **f), torch.empty(n, 4, **f),
                           torch.empty(n, **f), torch.empty(n, 4, device=device, dtype=torch.int16),
                           torch.empty(n, device=device, dtype=torch.int32))

    def c(self, rows: int | None = None) -> Proj:
        """Checked for `rows` Gaussians (default: the rows of `depth`)."""
        r = int(self.depth.shape[0]) if rows is None else int(rows)
        return Proj(_arr(self.xy, "proj.xy", F32, 4 * r), _arr(self.conic_opac, "proj.conic_opac", F32, 4 * r),
                    _arr(self.rgb, "proj.rgb", F32, 4 * r), _arr(self.depth, "proj.depth", F32, r),
                    _arr(self.rect, "proj.rect", I16, 4 * r), _arr(self.tiles_touched, "proj.tiles_touched", I32, r))


@dataclass
class BinBuffers:
    gids: torch.Tensor     # [cap] i32 (uint32 in C)
    keys: torch.Tensor | None  # [cap] i64 (uint64 in C) or None
    ranges: torch.Tensor   # [T,2] i32 (uint32 in C)
    count: torch.Tensor    # [1] i32
    capacity: int
    order: torch.Tensor | None = None   # [T] i32 (uint32 in C): tile schedule, longest lists first
    walk: torch.Tensor | None = None        # [W*cap] i32: the forward's walk lists (W warps per tile)
    walk_count: torch.Tensor | None = None  # [T*W] i32
    walk_warps: int = 0

    @staticmethod
    def alloc(capacity: int, num_tiles: int, with_keys=False, device="cuda", with_order=True,
              walk_warps: int = 0) -> "BinBuffers":
        """walk_warps > 0 (tile pixels / 32): room for the forward pass's walk
        lists, which the backward pass then follows."""
        i32 = dict(device=device, dtype=torch.int32)
        cap = max(capacity, 1)
        return BinBuffers(torch.empty(cap, **i32),
                          torch.empty(cap, device=device, dtype=torch.int64) if with_keys else None,
                          torch.empty(num_tiles, 2, **i32), torch.zeros(1, **i32), capacity,
                          torch.empty(max(num_tiles, 1), **i32) if with_order else None,
                          torch.empty(walk_warps * cap, **i32) if walk_warps else None,
                          torch.zeros(max(num_tiles * walk_warps, 1), **i32) if walk_warps else None, walk_warps)

    def c(self, num_tiles: int | None = None) -> Bins:
        """Checked for `capacity` instances and `num_tiles` tiles (default:
        the rows of `ranges`)."""
        T = int(self.ranges.shape[0]) if num_tiles is None else int(num_tiles)
        cap = int(self.capacity)
        Wn = int(self.walk_warps)
        return Bins(_arr(self.gids, "bins.gids", I32, cap), _arr(self.keys, "bins.keys", I64, cap),
                    _arr(self.ranges, "bins.ranges", I32, 2 * T), _arr(self.count, "bins.count", I32, 1), cap,
                    _arr(self.order, "bins.order", I32, T), _arr(self.walk, "bins.walk", I32, Wn * cap),
                    _arr(self.walk_count, "bins.walk_count", I32, T * Wn))

    def for_settings(self, st) -> "BinBuffers":
        """Checks that the walk lists were sized for the tile shape of `st`."""
        if self.walk is not None and self.walk_warps != st.tile_w * st.tile_h // 32:
            raise ValueError("bins: walk lists sized for another tile shape")
        return self


def camera_c(cam) -> Camera:
    """Marshals a camera with fields R (3x3), t (3), fx, fy, cx, cy, width, height, near_z."""
    R = [float(x) for x in torch.as_tensor(cam.R, dtype=torch.float32).reshape(-1).tolist()]
    t = [float(x) for x in torch.as_tensor(cam.t, dtype=torch.float32).reshape(-1).tolist()]
    return Camera((C.c_float * 9)(*R), (C.c_float * 3)(*t), cam.fx, cam.fy, cam.cx, cam.cy,
                  int(cam.width), int(cam.height), getattr(cam, "near_z", 0.2))


def settings_c(st) -> Settings:
    return Settings(st.tile_w, st.tile_h, st.alpha_min, st.alpha_max, st.T_min, st.radius_sigma,
                    st.dilation, st.fov_clamp, (C.c_float * 3)(*[float(x) for x in st.bg]))


def num_tiles(cam, st) -> int:
    return ((cam.width + st.tile_w - 1) // st.tile_w) * ((cam.height + st.tile_h - 1) // st.tile_h)


# --------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# --------------------------------------------------------------------------
def project(g: GaussianTensors, cam, st, out: ProjBuffers, stream=None):
    gc, cc, sc, oc = g.c(), camera_c(cam), settings_c(st), out.c(g.n)
    _check("sgs_project", lib().sgs_project(C.byref(gc), C.byref(cc), C.byref(sc), C.byref(oc), _stream(stream)))


def bin_sort_workspace_size(n: int, capacity: int, tiles: int) -> int:
    b = C.c_size_t()
    _check("sgs_bin_sort_workspace_size", lib().sgs_bin_sort_workspace_size(n, capacity, tiles, C.byref(b)))
    return b.value


def bin_sort(proj: ProjBuffers, n: int, cam, st, out: BinBuffers, ws: torch.Tensor, stream=None):
    pc, cc, sc, oc = proj.c(n), camera_c(cam), settings_c(st), out.c(num_tiles(cam, st))
    _check("sgs_bin_sort", lib().sgs_bin_sort(C.byref(pc), n, C.byref(cc), C.byref(sc), C.byref(oc), _p(ws),
                                               ws.numel() * ws.element_size(), _stream(stream)))


def render_fwd(proj: ProjBuffers, bins: BinBuffers, cam, st, image, final_T, n_contrib, stream=None):
    pc, bc, cc, sc = proj.c(), bins.for_settings(st).c(num_tiles(cam, st)), camera_c(cam), settings_c(st)
    P = _pixels(cam)
    _check("sgs_render_fwd", lib().sgs_render_fwd(C.byref(pc), C.byref(bc), C.byref(cc), C.byref(sc),
                                                   _arr(image, "image", F32, 3 * P),
                                                   _arr(final_T, "final_T", F32, P),
                                                   _arr(n_contrib, "n_contrib", I32, P), _stream(stream)))


def render_fwd_l1(proj: ProjBuffers, bins: BinBuffers, cam, st, target, n_views: int, image, final_T, n_contrib,
                  dL_dimage, loss, stream=None):
    """render_fwd with the L1 loss and its gradient in the same kernel."""
    pc, bc, cc, sc = proj.c(), bins.for_settings(st).c(num_tiles(cam, st)), camera_c(cam), settings_c(st)
    P = _pixels(cam)
    _check("sgs_render_fwd_l1", lib().sgs_render_fwd_l1(C.byref(pc), C.byref(bc), C.byref(cc), C.byref(sc),
                                                         _arr(target, "target", F32, 3 * P), int(n_views),
                                                         _arr(image, "image", F32, 3 * P),
                                                         _arr(final_T, "final_T", F32, P),
                                                         _arr(n_contrib, "n_contrib", I32, P),
                                                         _arr(dL_dimage, "dL_dimage", F32, 3 * P),
                                                         _arr(loss, "loss", F32, 1), _stream(stream)))


def render_stats(proj: ProjBuffers, bins: BinBuffers, cam, st, counts, stream=None, warp_union=None):
    """counts: int32 [H,W,2] <- (pairs evaluated, pairs composited) per pixel;
    warp_union (optional) int32 [T * tile pixels / 32] <- per 8x4 block, the
    list entries at least one of its pixels composites."""
    pc, bc, cc, sc = proj.c(), bins.for_settings(st).c(num_tiles(cam, st)), camera_c(cam), settings_c(st)
    nw = num_tiles(cam, st) * (st.tile_w * st.tile_h // 32)
    _check("sgs_render_stats", lib().sgs_render_stats(C.byref(pc), C.byref(bc), C.byref(cc), C.byref(sc),
                                                       _arr(counts, "counts", I32, 2 * _pixels(cam)),
                                                       _arr(warp_union, "warp_union", I32, nw), _stream(stream)))


def ssim_l1_workspace_size(height: int, width: int) -> int:
    b = C.c_size_t()
    _check("sgs_ssim_l1_workspace_size", lib().sgs_ssim_l1_workspace_size(int(height), int(width), C.byref(b)))
    return b.value


def ssim_l1_loss_grad(image, target, n_views: int, lambda_dssim: float, dL_dimage, loss, ws, stream=None):
    """loss += ((1 - lambda) L1 + lambda (1 - SSIM)) / n_views; dL_dimage <- its gradient."""
    H, W = _image_hw(image)
    _check("sgs_ssim_l1_loss_grad",
           lib().sgs_ssim_l1_loss_grad(_arr(image, "image", F32, 3 * H * W), _arr(target, "target", F32, 3 * H * W),
                                       H, W, n_views, float(lambda_dssim),
                                       _arr(dL_dimage, "dL_dimage", F32, 3 * H * W), _arr(loss, "loss", F32, 1),
                                       _p(ws), ws.numel() * ws.element_size(), _stream(stream)))


def fma_probe(out, blocks: int, iters: int, stream=None):
    """FP32 FMA throughput probe: out float32 [blocks * 256]; 16 * iters FLOP
    per thread."""
    _check("sgs_fma_probe", lib().sgs_fma_probe(_arr(out, "out", F32, int(blocks) * 256), int(blocks), int(iters),
                                                 _stream(stream)))


def _image_hw(image) -> tuple[int, int]:
    if not isinstance(image, torch.Tensor) or image.dim() != 3 or image.shape[2] != 3:
        raise ValueError("image: expected a [H, W, 3] tensor")
    return int(image.shape[0]), int(image.shape[1])


def l1_loss_grad(image, target, n_views: int, dL_dimage, loss, stream=None):
    H, W = _image_hw(image)
    _check("sgs_l1_loss_grad", lib().sgs_l1_loss_grad(_arr(image, "image", F32, 3 * H * W),
                                                       _arr(target, "target", F32, 3 * H * W), H, W, n_views,
                                                       _arr(dL_dimage, "dL_dimage", F32, 3 * H * W),
                                                       _arr(loss, "loss", F32, 1), _stream(stream)))


def render_bwd_workspace_size(n: int) -> int:
    b = C.c_size_t()
    _check("sgs_render_bwd_workspace_size", lib().sgs_render_bwd_workspace_size(n, C.byref(b)))
    return b.value


BWD_ACCUMULATE_GRADS, BWD_RESET_S = 1, 2


def _bwd_flags(accumulate: bool, reset_S: bool) -> int:
    return (BWD_ACCUMULATE_GRADS if accumulate else 0) | (BWD_RESET_S if reset_S else 0)


def clear(t: torch.Tensor, stream=None):
    """Zeroes a contiguous device tensor with a memset on `stream` (no kernel)."""
    if not t.is_contiguous():
        raise ValueError("clear: tensor must be contiguous")
    _check("sgs_clear", lib().sgs_clear(_p(t), t.numel() * t.element_size(), _stream(stream)))


def render_bwd_with_splitting(g: GaussianTensors, proj: ProjBuffers, bins: BinBuffers, cam, st, final_T,
                              n_contrib, dL_dimage, grads: GaussianTensors, S_accum, ws, stream=None,
                              accumulate: bool = True, S_po=None, S_ls=None, reset_S: bool = False):
    """S_po [N,3] (optional): the position-opacity block of the splitting
    matrix over theta = (p, o) is accumulated too; S_ls [N,18] (optional, with
    S_po): the log-scale blocks over theta = (p, l, o) as well.  reset_S: the
    call starts a new accumulation period (S, S_po, S_ls overwritten)."""
    gc, pc, bc, cc, sc = g.c(), proj.c(g.n), bins.for_settings(st).c(num_tiles(cam, st)), camera_c(cam), \
        settings_c(st)
    grc = grads.grads_c(g)
    n, P = g.n, _pixels(cam)
    _check("sgs_render_bwd_with_splitting",
           lib().sgs_render_bwd_with_splitting(C.byref(gc), C.byref(pc), C.byref(bc), C.byref(cc), C.byref(sc),
                                               _arr(final_T, "final_T", F32, P), _arr(n_contrib, "n_contrib", I32, P),
                                               _arr(dL_dimage, "dL_dimage", F32, 3 * P), C.byref(grc),
                                               _bwd_flags(accumulate, reset_S), _arr(S_accum, "S_accum", F32, 6 * n),
                                               _arr(S_po, "S_po", F32, 3 * n), _arr(S_ls, "S_ls", F32, 18 * n), _p(ws),
                                               ws.numel() * ws.element_size(),
                                               _stream(stream)))


def cameras_c(cams):
    arr = (Camera * len(cams))()
    for k, c in enumerate(cams):
        arr[k] = camera_c(c)
    return arr


def render_views_workspace_size(n: int, cams, st, capacity: int) -> int:
    b = C.c_size_t()
    arr, sc = cameras_c(cams), settings_c(st)
    _check("sgs_render_views_workspace_size",
           lib().sgs_render_views_workspace_size(n, arr, len(cams), C.byref(sc), capacity, C.byref(b)))
    return b.value


def render_views_with_splitting(g: GaussianTensors, cams, st, batch: int, targets, images, loss,
                                grads: GaussianTensors, accumulate: bool, S_accum, d_count, capacity: int, ws,
                                stream=None, S_po=None, reset_S: bool = False):
    """All views in one pass: project, bin/sort, persistent forward, L1,
    persistent backward, projection adjoint (see sgs_render_views_with_splitting);
    reset_S: S (and S_po) overwritten instead of added to."""
    gc, arr, sc = g.c(), cameras_c(cams), settings_c(st)
    grc = grads.grads_c(g)
    n, P = g.n, sum(_pixels(c) for c in cams)
    _check("sgs_render_views_with_splitting",
           lib().sgs_render_views_with_splitting(C.byref(gc), arr, len(cams), C.byref(sc), batch,
                                                 _arr(targets, "targets", F32, 3 * P),
                                                 _arr(images, "images", F32, 3 * P), _arr(loss, "loss", F32, 1),
                                                 C.byref(grc), _bwd_flags(accumulate, reset_S),
                                                 _arr(S_accum, "S_accum", F32, 6 * n), _arr(S_po, "S_po", F32, 3 * n),
                                                 _arr(d_count, "d_count", I32, 1), capacity, _p(ws),
                                                 ws.numel() * ws.element_size(), _stream(stream)))


def render_views_bins(n: int, cams, st, capacity: int, ws: torch.Tensor, count: torch.Tensor) -> BinBuffers:
    """The binning the last render_views_with_splitting call left in `ws`
    (gids = projection rows v*n + i, ranges over global tile ids), as tensor
    views into ws (valid while ws holds that call's results)."""
    arr, sc = cameras_c(cams), settings_c(st)
    b = Bins()
    _check("sgs_render_views_bins",
           lib().sgs_render_views_bins(n, arr, len(cams), C.byref(sc), capacity, _p(ws),
                                       ws.numel() * ws.element_size(), C.byref(b)))
    T = sum(num_tiles(c, st) for c in cams)
    base = ws.data_ptr()
    nbytes = ws.numel() * ws.element_size()

    def view(ptr, count_):
        off = int(ptr) - base
        if off < 0 or off + 4 * count_ > nbytes:
            raise RuntimeError("sgs_render_views_bins: pointer outside the workspace")
        return ws[off:off + 4 * count_].view(torch.int32)

    return BinBuffers(view(b.gids, max(capacity, 1)), None, view(b.ranges, 2 * T).view(T, 2), count, capacity,
                      view(b.order, max(T, 1)))


def _scenes_c(scenes):
    arr = (Gaussians * len(scenes))()
    for k, g in enumerate(scenes):
        arr[k] = g.c()
    return arr


def render_batch_workspace_size(scenes, cams, st, capacity: int) -> int:
    b = C.c_size_t()
    sa, ca, sc = _scenes_c(scenes), cameras_c(cams), settings_c(st)
    _check("sgs_render_batch_workspace_size",
           lib().sgs_render_batch_workspace_size(sa, ca, len(cams), C.byref(sc), capacity, C.byref(b)))
    return b.value


def render_batch_fwd(scenes, cams, st, batch: int, images, d_count, capacity: int, ws, stream=None):
    """Forward render of views of (possibly different) scenes in one pass."""
    sa, ca, sc = _scenes_c(scenes), cameras_c(cams), settings_c(st)
    P = sum(_pixels(c) for c in cams)
    _check("sgs_render_batch_fwd",
           lib().sgs_render_batch_fwd(sa, ca, len(cams), C.byref(sc), batch, _arr(images, "images", F32, 3 * P),
                                      _arr(d_count, "d_count", I32, 1), capacity,
                                      _p(ws), ws.numel() * ws.element_size(), _stream(stream)))


def adam_step(param, grad, m, v, lr: float, step: int, beta1=0.9, beta2=0.999, eps=1e-8, grad_accum=None,
              stream=None):
    """In-place Adam update of one float32 parameter tensor."""
    k = param.numel()
    _check("sgs_adam_step", lib().sgs_adam_step(_arr(param, "param", F32), _arr(grad, "grad", F32, k),
                                                 _arr(m, "m", F32, k), _arr(v, "v", F32, k), k, lr, beta1, beta2,
                                                 eps, step, _arr(grad_accum, "grad_accum", F32, k), _stream(stream)))


def adam_step_dev(param, grad, m, v, lr: float, d_step, beta1=0.9, beta2=0.999, eps=1e-8, grad_accum=None,
                  stream=None):
    """adam_step with the step count read from the device int32 tensor d_step."""
    k = param.numel()
    _check("sgs_adam_step_dev", lib().sgs_adam_step_dev(_arr(param, "param", F32), _arr(grad, "grad", F32, k),
                                                         _arr(m, "m", F32, k), _arr(v, "v", F32, k), k, lr, beta1,
                                                         beta2, eps, _arr(d_step, "d_step", I32, 1),
                                                         _arr(grad_accum, "grad_accum", F32, k), _stream(stream)))


def _split_arrays(n, S_accum, S_po, S_ls):
    return (_arr(S_accum, "S_accum", F32, 6 * n), _arr(S_po, "S_po", F32, 3 * n), _arr(S_ls, "S_ls", F32, 18 * n))


def _split_outputs(n, capacity, S_po, S_ls, d_n_out, parent_index, lam_min_out, v_min_out):
    d = 7 if S_ls is not None else (4 if S_po is not None else 3)
    return (_arr(d_n_out, "d_n_out", I32, 1), _arr(parent_index, "parent_index", I32, capacity),
            _arr(lam_min_out, "lam_min_out", F32, n), _arr(v_min_out, "v_min_out", F32, d * n))


def densify_split_workspace_size(n: int) -> int:
    b = C.c_size_t()
    _check("sgs_densify_split_workspace_size", lib().sgs_densify_split_workspace_size(n, C.byref(b)))
    return b.value


def densify_split(g: GaussianTensors, S_accum, inv_T_split: float, eps_split: float, step_scale: float,
                  grad_norm, eps_grad: float, out: GaussianTensors, capacity: int, d_n_out, parent_index,
                  lam_min_out, v_min_out, ws, stream=None, max_splits: int = 0, S_po=None, S_ls=None):
    """S_po [N,3] given: split over theta = (p, o) (v_min_out [N,4]); S_po and
    S_ls [N,18] given: over theta = (p, l, o) (v_min_out [N,7])."""
    gc, oc = g.c(), out.c_mut(capacity)
    _check("sgs_densify_split",
           lib().sgs_densify_split(C.byref(gc), *_split_arrays(g.n, S_accum, S_po, S_ls), inv_T_split,
                                   eps_split, step_scale, _arr(grad_norm, "grad_norm", F32, g.n), eps_grad,
                                   int(max_splits), C.byref(oc), capacity,
                                   *_split_outputs(g.n, capacity, S_po, S_ls, d_n_out, parent_index, lam_min_out,
                                                   v_min_out), _p(ws), ws.numel() * ws.element_size(),
                                   _stream(stream)))


def kernel_launches() -> int:
    """Kernel launches issued by the library so far (process-wide)."""
    return int(lib().sgs_kernel_launches())


def densify_split_noalloc(g: GaussianTensors, S_accum, inv_T_split: float, eps_split: float, step_scale: float,
                          grad_norm, eps_grad: float, out: GaussianTensors, capacity: int, d_n_out, parent_index,
                          lam_min_out, v_min_out, stream=None, max_splits: int = 0, S_po=None, S_ls=None):
    """densify_split without a workspace, for callers that cannot allocate one
    (its scratch is a fixed array inside the library; n <= 1,000,000; calls
    that overlap on the GPU race)."""
    gc, oc = g.c(), out.c_mut(capacity)
    _check("sgs_densify_split_noalloc",
           lib().sgs_densify_split_noalloc(C.byref(gc), *_split_arrays(g.n, S_accum, S_po, S_ls),
                                           inv_T_split, eps_split, step_scale,
                                           _arr(grad_norm, "grad_norm", F32, g.n), eps_grad, int(max_splits),
                                           C.byref(oc), capacity,
                                           *_split_outputs(g.n, capacity, S_po, S_ls, d_n_out, parent_index,
                                                           lam_min_out, v_min_out), _stream(stream)))


def check_count(M: int) -> int:
    """Instance count read back from bin_sort / the batched entry points
    (never negative; a negative value means corrupted device state)."""
    if M < 0:
        raise RuntimeError(f"sgs_bin_sort: invalid instance count {M}")
    return M


def workspace(nbytes: int, device="cuda") -> torch.Tensor:
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)
