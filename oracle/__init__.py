"""CPU oracle for the SteepGS splitting path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it, and
the two share no code: this wrapper drives ``steepgs_oracle.c`` (plain C,
float64 for continuous quantities, compiled with ``-ffp-contract=off``).

Every function cites the passage of the paper it follows in the C source.
Inputs come from ``synth`` (seeded generators that hold none of the method's
arithmetic).  ``oracle.ssim`` (plain float64 numpy) holds the SSIM term of the
loss.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "steepgs_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction, so float32 sums are exact IEEE sequences)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-fopenmp",
               "-shared", "-o", tmp, _SRC, "-lm"]
        if subprocess.run(cmd).returncode != 0:          # no OpenMP: the all-core variants run on one thread
            subprocess.run([c for c in cmd if c != "-fopenmp"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Scene(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int32),
                ("sh_degree", C.c_int32)]


class _Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("near_z", C.c_float)]


class _Settings(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("alpha_min", C.c_float),
                ("alpha_max", C.c_float), ("T_min", C.c_float), ("radius_sigma", C.c_float),
                ("dilation", C.c_float), ("fov_clamp", C.c_float), ("bg", C.c_float * 3)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P = C.c_void_p
            lib.orc_exp_f32_export.restype = C.c_float
            lib.orc_exp_f32_export.argtypes = [C.c_float]
            lib.orc_integer_stage.argtypes = [P, P, P, P, P, P, P]
            lib.orc_project.argtypes = [P, P, P, P, P, P, P, P, P, P]
            lib.orc_bin_sort.restype = C.c_int64
            lib.orc_bin_sort.argtypes = [P, P, P, P, P, P, C.c_int64]
            lib.orc_render.argtypes = [P, P, P, P, P, P, P]
            lib.orc_render_rows.argtypes = [P, P, P, C.c_int, C.c_int, P, P, P, P]
            lib.orc_backward_rows.argtypes = [P, P, P, C.c_int, C.c_int, P, P, P, P, P, P, P, P, P, P]
            lib.orc_render_rows_mt.argtypes = lib.orc_render_rows.argtypes
            lib.orc_backward_rows_mt.argtypes = lib.orc_backward_rows.argtypes
            lib.orc_threads.restype = C.c_int
            lib.orc_l1_loss_grad.restype = C.c_double
            lib.orc_l1_loss_grad.argtypes = [P, P, C.c_int, C.c_int, C.c_int, P]
            lib.orc_backward.argtypes = [P, P, P, P, P, P, P, P, P, P, P, P, P]
            lib.orc_frozen_eval.restype = C.c_double
            lib.orc_frozen_eval.argtypes = [P, P, P, C.c_int, P, P, C.c_int, P, P, C.c_double, P]
            lib.orc_eig3_min.argtypes = [P, C.c_double, C.c_int, P, P]
            lib.orc_jacobi3.argtypes = [P, C.c_int, P, P]
            lib.orc_split.restype = C.c_int
            lib.orc_split.argtypes = [P, P, P, C.c_double, C.c_double, P, C.c_double, C.c_int64,
                                      P, P, P, P, P, P, P, P]
            lib.orc_sh_basis.argtypes = [C.c_int, P, C.c_int, P, P]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class _Bound:
    """Keeps the numpy arrays behind the ctypes structs alive."""

    def __init__(self, scene, cam, st):
        self.arrs = [np.ascontiguousarray(scene.means, np.float32),
                     np.ascontiguousarray(scene.log_scales, np.float32),
                     np.ascontiguousarray(scene.quats, np.float32),
                     np.ascontiguousarray(scene.opacity_logit, np.float32),
                     np.ascontiguousarray(scene.sh, np.float32)]
        a = self.arrs
        self.scene = _Scene(_ptr(a[0]), _ptr(a[1]), _ptr(a[2]), _ptr(a[3]), _ptr(a[4]),
                            int(a[0].shape[0]), int(scene.sh_degree))
        self.cam = None
        if cam is not None:
            self.cam = _Camera((C.c_float * 9)(*np.asarray(cam.R, np.float32).reshape(-1).tolist()),
                               (C.c_float * 3)(*np.asarray(cam.t, np.float32).tolist()),
                               cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height, cam.near_z)
        self.st = None
        if st is not None:
            self.st = _Settings(st.tile_w, st.tile_h, st.alpha_min, st.alpha_max, st.T_min,
                                st.radius_sigma, st.dilation, st.fov_clamp,
                                (C.c_float * 3)(*[float(x) for x in st.bg]))

    def refs(self):
        return (C.byref(self.scene), C.byref(self.cam) if self.cam is not None else None,
                C.byref(self.st) if self.st is not None else None)


def n_tiles(cam, st):
    gx = (cam.width + st.tile_w - 1) // st.tile_w
    gy = (cam.height + st.tile_h - 1) // st.tile_h
    return gx, gy


def exp_f32(x):
    lib = _load()
    x = np.asarray(x, np.float32).reshape(-1)
    return np.array([lib.orc_exp_f32_export(float(v)) for v in x], np.float32)


def sh_basis(degree, dirs):
    lib = _load()
    dirs = np.ascontiguousarray(dirs, np.float64)
    n = dirs.shape[0]
    K = (degree + 1) ** 2
    Y = np.zeros((n, K))
    dY = np.zeros((n, K, 3))
    lib.orc_sh_basis(degree, _ptr(dirs), n, _ptr(Y), _ptr(dY))
    return Y, dY


def integer_stage(scene, cam, st):
    """Float32 integer stage: 2-D mean, depth, inclusive tile rect, tile count."""
    lib = _load()
    b = _Bound(scene, cam, st)
    n = scene.n
    mean2d = np.zeros((n, 2), np.float32)
    depth = np.zeros(n, np.float32)
    rect = np.zeros((n, 4), np.int32)
    tiles = np.zeros(n, np.int32)
    lib.orc_integer_stage(*b.refs(), _ptr(mean2d), _ptr(depth), _ptr(rect), _ptr(tiles))
    return dict(mean2d=mean2d, depth=depth, rect=rect, tiles=tiles)


def project(scene, cam, st):
    """Float64 projected state per Gaussian (Section 3, Eq. sigma_2D)."""
    lib = _load()
    b = _Bound(scene, cam, st)
    n = scene.n
    out = dict(mean2d=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n),
               rgb=np.zeros((n, 3)), P=np.zeros((n, 2, 3)), depth=np.zeros(n),
               tiles=np.zeros(n, np.int32))
    lib.orc_project(*b.refs(), _ptr(out["mean2d"]), _ptr(out["conic"]), _ptr(out["opacity"]),
                    _ptr(out["rgb"]), _ptr(out["P"]), _ptr(out["depth"]), _ptr(out["tiles"]))
    return out


def bin_sort(scene, cam, st):
    """Instances ordered by (tile, float32 depth bits, gid); per-tile [start, end)."""
    lib = _load()
    b = _Bound(scene, cam, st)
    M = lib.orc_bin_sort(*b.refs(), None, None, None, 0)
    gx, gy = n_tiles(cam, st)
    keys = np.zeros(max(M, 1), np.uint64)
    gids = np.zeros(max(M, 1), np.uint32)
    ranges = np.zeros((gx * gy, 2), np.uint32)
    lib.orc_bin_sort(*b.refs(), _ptr(keys), _ptr(gids), _ptr(ranges), M)
    return keys[:M], gids[:M], ranges


def threads() -> int:
    """Host threads the all-core variants use (OpenMP; 1 without it)."""
    return int(_load().orc_threads())


def render(scene, cam, st, rows=None, all_cores=False):
    """Front-to-back compositing (Section 3, Eq. alpha_blend), float64.
    rows = (y0, h): only rows [y0, y0 + h) of the same view ([h, W] outputs).
    all_cores: the same per-pixel computation with rows dealt to all host
    threads (identical results; a timing baseline)."""
    lib = _load()
    b = _Bound(scene, cam, st)
    y0, H = (0, cam.height) if rows is None else rows
    W = cam.width
    image = np.zeros((H, W, 3))
    final_T = np.zeros((H, W))
    n_contrib = np.zeros((H, W), np.int32)
    band = np.zeros((H, W), np.uint8)
    fn = lib.orc_render_rows_mt if all_cores else lib.orc_render_rows
    if fn(*b.refs(), int(y0), int(H), _ptr(image), _ptr(final_T), _ptr(n_contrib), _ptr(band)) != 0:
        raise ValueError("rows outside the view")
    return dict(image=image, final_T=final_T, n_contrib=n_contrib, band=band.astype(bool))


def l1_loss_grad(image, target, n_views=1):
    """L1 photometric loss (Section 3, Eq. loss) and dL/dC."""
    lib = _load()
    image = np.ascontiguousarray(image, np.float64)
    target = np.ascontiguousarray(target, np.float32)
    H, W = image.shape[:2]
    g = np.zeros_like(image)
    L = lib.orc_l1_loss_grad(_ptr(image), _ptr(target), H, W, n_views, _ptr(g))
    return L, g


def backward(scene, cam, st, dL_dC, acc=None, rows=None, all_cores=False, blocks=True):
    """Parameter gradients and full 3x3 splitting matrices of one view
    (Section 4.4, Algorithm 1), plus S_po [n,3], the position-opacity block of
    the splitting matrix over theta = (p, o).  Accumulates into `acc` when given.
    rows = (y0, h): only rows [y0, y0 + h) of the same view carry gradient
    (dL_dC is [h, W, 3]).  all_cores: rows dealt to all host threads, each
    summing into its own copy, the copies added at the end (the same terms in
    another order; a timing baseline).  blocks=False leaves out S_po and S_ls
    (the splitting matrix over the position only, as the paper's experiments)."""
    lib = _load()
    b = _Bound(scene, cam, st)
    n, K = scene.n, (scene.sh_degree + 1) ** 2
    if acc is None:
        acc = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
                   opacity_logit=np.zeros(n), sh=np.zeros((n, K, 3)), S=np.zeros((n, 3, 3)),
                   S_po=np.zeros((n, 3)), S_ls=np.zeros((n, 18)))
    grad2d = np.zeros((n, 9))
    dL = np.ascontiguousarray(dL_dC, np.float64)
    y0, h = (0, cam.height) if rows is None else rows
    if dL.shape[:2] != (h, cam.width):
        raise ValueError("dL_dC must cover the rows")
    fn = lib.orc_backward_rows_mt if all_cores else lib.orc_backward_rows
    if fn(*b.refs(), int(y0), int(h), _ptr(dL), _ptr(acc["means"]), _ptr(acc["log_scales"]),
          _ptr(acc["quats"]), _ptr(acc["opacity_logit"]), _ptr(acc["sh"]),
          _ptr(acc["S"]), _ptr(acc["S_po"] if blocks else None), _ptr(acc["S_ls"] if blocks else None),
          _ptr(grad2d)) != 0:
        raise ValueError("rows outside the view")
    acc["grad2d"] = grad2d
    return acc


def frozen_eval(scene, cam, st, idx, dp=None, mix_v=None, g=None, target=None, d_o=0.0, d_ls=None):
    """Loss in the frozen-linearisation model (Appendix "Deriving Hessian of
    Gaussian") with Gaussian `idx` displaced by dp (opacity by d_o) or replaced
    by the w = 1/2 mixture slot at (p +- mix_v, o +- d_o, log-scales +- d_ls;
    P frozen).  Returns sum g.C (g given) or the L1 loss."""
    lib = _load()
    b = _Bound(scene, cam, st)
    mode = 0 if g is not None else 1
    g_arr = None if g is None else np.ascontiguousarray(g, np.float64)
    t_arr = None if target is None else np.ascontiguousarray(target, np.float32)
    dp_arr = None if dp is None else np.ascontiguousarray(dp, np.float64)
    mv_arr = None if mix_v is None else np.ascontiguousarray(mix_v, np.float64)
    ls_arr = None if d_ls is None else np.ascontiguousarray(d_ls, np.float64)
    return lib.orc_frozen_eval(*b.refs(), mode, _ptr(g_arr), _ptr(t_arr), int(idx),
                               _ptr(dp_arr), _ptr(mv_arr), float(d_o), _ptr(ls_arr))


def eig3_min(S, scale=1.0):
    """Minimum eigenpair by the trigonometric root formula (Appendix "Eigendecomposition")."""
    lib = _load()
    S = np.ascontiguousarray(S, np.float64).reshape(-1, 9)
    n = S.shape[0]
    lam = np.zeros(n)
    v = np.zeros((n, 3))
    lib.orc_eig3_min(_ptr(S), float(scale), n, _ptr(lam), _ptr(v))
    return lam, v


def jacobi3(S):
    """All eigenpairs by cyclic Jacobi rotations (independent cross-check)."""
    lib = _load()
    S = np.ascontiguousarray(S, np.float64).reshape(-1, 9)
    n = S.shape[0]
    ev = np.zeros((n, 3))
    V = np.zeros((n, 3, 3))
    lib.orc_jacobi3(_ptr(S), n, _ptr(ev), _ptr(V))
    return ev, V


def split(scene, lam, v, eps_split, step_scale=1.0, grad_norm=None, eps_grad=0.0, budget=0, flags=None):
    """Steepest density control split and compaction (Theorem 2, Algorithm 1);
    budget > 0 keeps only the `budget` least lambda_min (Variants section).
    `flags` (bool [n]), when given, replaces the split rule: the exclusive
    scan, parent indices and offspring follow from those decisions."""
    lib = _load()
    b = _Bound(scene, None, None)
    n, K = scene.n, (scene.sh_degree + 1) ** 2
    cap = 2 * n
    out = dict(means=np.zeros((cap, 3)), log_scales=np.zeros((cap, 3)), quats=np.zeros((cap, 4)),
               opacity_logit=np.zeros(cap), sh=np.zeros((cap, K, 3)),
               parent=np.zeros(cap, np.int32))
    flags_in, flags = flags, np.zeros(n, np.uint8)
    lam = np.ascontiguousarray(lam, np.float64)
    v = np.ascontiguousarray(v, np.float64)
    gn = None if grad_norm is None else np.ascontiguousarray(grad_norm, np.float64)
    f_in = None if flags_in is None else np.ascontiguousarray(np.asarray(flags_in, bool).astype(np.uint8))
    if f_in is not None and f_in.shape != (n,):
        raise ValueError("flags must hold one decision per Gaussian")
    n_out = lib.orc_split(C.byref(b.scene), _ptr(lam), _ptr(v), float(eps_split), float(step_scale),
                          _ptr(gn), float(eps_grad), int(budget), _ptr(out["means"]), _ptr(out["log_scales"]),
                          _ptr(out["quats"]), _ptr(out["opacity_logit"]), _ptr(out["sh"]),
                          _ptr(out["parent"]), _ptr(flags), _ptr(f_in))
    for k in list(out):
        out[k] = out[k][:n_out]
    out["flags"] = flags.astype(bool)
    out["n_out"] = n_out
    return out


def S4_matrix(S, S_po):
    """Splitting matrices over theta = (p, o) (dim Theta = 4): [[S_pp, S_po],
    [S_po^T, 0]], the opacity-opacity entry being d^2 sigma / do^2 = 0."""
    S = np.asarray(S, np.float64)
    S_po = np.asarray(S_po, np.float64)
    n = S.shape[0]
    S4 = np.zeros((n, 4, 4))
    S4[:, :3, :3] = S
    S4[:, :3, 3] = S_po
    S4[:, 3, :3] = S_po
    return S4


def eig_min_sym(S, scale=1.0):
    """Minimum eigenpair of symmetric matrices [n, d, d] (d small) by LAPACK's
    symmetric solver; eigenvector sign: the component of largest magnitude is
    positive (lowest index on ties)."""
    w, V = np.linalg.eigh(np.asarray(S, np.float64) * scale)
    lam = w[:, 0].copy()
    v = V[:, :, 0].copy()
    k = np.argmax(np.abs(v), axis=1)
    sgn = np.where(v[np.arange(len(v)), k] < 0, -1.0, 1.0)
    return lam, v * sgn[:, None]


def S7_matrix(S, S_po, S_ls):
    """Splitting matrices over theta = (p, l, o) (dim Theta = 7, l the
    log-scales): blocks p-p (S), p-l (S_ls[:, :9], row p), l-l (S_ls[:, 9:15],
    xx xy xz yy yz zz), p-o (S_po), l-o (S_ls[:, 15:18]), o-o = 0."""
    S = np.asarray(S, np.float64)
    n = S.shape[0]
    S7 = np.zeros((n, 7, 7))
    S7[:, :3, :3] = S
    pl = np.asarray(S_ls, np.float64)[:, :9].reshape(n, 3, 3)
    S7[:, :3, 3:6] = pl
    S7[:, 3:6, :3] = np.transpose(pl, (0, 2, 1))
    iu = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for q, (a, b) in enumerate(iu):
        S7[:, 3 + a, 3 + b] = S_ls[:, 9 + q]
        S7[:, 3 + b, 3 + a] = S_ls[:, 9 + q]
    S7[:, :3, 6] = S_po
    S7[:, 6, :3] = S_po
    S7[:, 3:6, 6] = S_ls[:, 15:18]
    S7[:, 6, 3:6] = S_ls[:, 15:18]
    return S7


OPACITY_SPLIT_MIN, OPACITY_SPLIT_MAX = 1e-4, 1.0 - 1e-4


def split_po(scene, lam, v4, eps_split, step_scale=1.0, flags=None):
    """Steepest split over theta = (p, o) (v4 [n, 4]) or (p, l, o) (v [n, 7],
    l the log-scales): Gaussian i with lambda_min < eps_split becomes the
    w = 1/2 pair at theta +- eps_i v, eps_i = step_scale * max_k
    exp(log_scale_ik); each offspring keeps half of its displaced opacity,
    (o +- eps_i v_o) / 2 clamped to [1e-4, 1 - 1e-4]; the parent's row takes
    the + offspring, the - offspring is appended in index order.  `flags`
    (bool [n]), when given, replaces the rule lambda_min < eps_split."""
    n = scene.n
    K = (scene.sh_degree + 1) ** 2
    flags = np.asarray(lam) < eps_split if flags is None else np.asarray(flags, bool).copy()
    if flags.shape != (n,):
        raise ValueError("flags must hold one decision per Gaussian")
    idx = np.nonzero(flags)[0]
    n_out = n + len(idx)
    eps = step_scale * np.exp(scene.log_scales.astype(np.float64)).max(axis=1)
    o = 1.0 / (1.0 + np.exp(-scene.opacity_logit.astype(np.float64)))
    out = dict(means=np.zeros((n_out, 3)), log_scales=np.zeros((n_out, 3)), quats=np.zeros((n_out, 4)),
               opacity_logit=np.zeros(n_out), sh=np.zeros((n_out, K, 3)), parent=np.zeros(n_out, np.int32))
    rows_p = np.arange(n)
    out["means"][:n] = scene.means
    out["log_scales"][:n] = scene.log_scales
    out["quats"][:n] = scene.quats
    out["opacity_logit"][:n] = scene.opacity_logit
    out["sh"][:n] = scene.sh
    out["parent"][:n] = rows_p
    v4 = np.asarray(v4, np.float64)
    for r, i in enumerate(idx):
        j = n + r
        for row, sgn in ((i, 1.0), (j, -1.0)):
            out["means"][row] = scene.means[i].astype(np.float64) + sgn * eps[i] * v4[i, :3]
            oj = np.clip(0.5 * (o[i] + sgn * eps[i] * v4[i, -1]), OPACITY_SPLIT_MIN, OPACITY_SPLIT_MAX)
            out["opacity_logit"][row] = np.log(oj) - np.log1p(-oj)
            out["log_scales"][row] = scene.log_scales[i].astype(np.float64) + (
                sgn * eps[i] * v4[i, 3:6] if v4.shape[1] == 7 else 0.0)
            out["quats"][row] = scene.quats[i]
            out["sh"][row] = scene.sh[i]
            out["parent"][row] = i
    out["flags"] = flags
    out["n_out"] = n_out
    return out


def densify_iteration(scene, cams, st, targets, T_split=1.0, eps_split=0.0, step_scale=1.0):
    """One fused iteration over the given views: render, L1 loss, backward with
    splitting matrices (summed over views), eigenpairs, split.  Used by the
    CPU-baseline timing and by end-to-end parity tests."""
    acc = None
    loss = 0.0
    V = len(cams)
    for cam, tgt in zip(cams, targets):
        r = render(scene, cam, st)
        L, g = l1_loss_grad(r["image"], tgt, V)
        loss += L
        acc = backward(scene, cam, st, g, acc)
    lam, v = eig3_min(acc["S"], 1.0 / T_split)
    sp = split(scene, lam, v, eps_split, step_scale)
    return dict(loss=loss, grads=acc, lam=lam, v=v, split=sp)
