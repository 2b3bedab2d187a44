"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed-form
colours, hand-composited pixels, brute-force enumeration, library routines,
finite differences, and the second-order statements of Theorems 1 and 2.
"""
import math

import numpy as np
import pytest

import oracle
import synth

SQRT_PI = math.sqrt(math.pi)


def _one_gaussian(mean, log_scale, logit, dc, quat=(1.0, 0.0, 0.0, 0.0)):
    n = np.asarray(mean).reshape(-1, 3).shape[0]
    return synth.Scene(np.asarray(mean, np.float32).reshape(n, 3),
                       np.asarray(log_scale, np.float32).reshape(n, 3),
                       np.broadcast_to(np.asarray(quat, np.float32).reshape(-1, 4), (n, 4)).copy(),
                       np.asarray(logit, np.float32).reshape(n),
                       np.asarray(dc, np.float32).reshape(n, 1, 3), 0)


# --------------------------------------------------------------------------
# Building blocks
# --------------------------------------------------------------------------

def test_exp_f32_within_two_ulp():
    """The float32 exponential of the integer stage is accurate (Cody-Waite +
    Taylor): within 2 ulp of the correctly rounded value."""
    x = np.concatenate([np.linspace(-20, 5, 20001), np.random.default_rng(0).normal(-9, 2, 5000)])
    x = x.astype(np.float32)
    got = oracle.exp_f32(x)
    ref = np.exp(x.astype(np.float64)).astype(np.float32)
    ulp = np.abs(got.view(np.int32).astype(np.int64) - ref.view(np.int32).astype(np.int64))
    assert ulp.max() <= 2


def test_sh_basis_orthonormal_and_gradient():
    """Real SH basis up to degree 3 is orthonormal on the sphere (Gauss-Legendre
    x uniform-phi quadrature, exact for these polynomial degrees) and its
    gradient matches central differences."""
    ct, wt = np.polynomial.legendre.leggauss(12)
    phis = np.linspace(0, 2 * np.pi, 24, endpoint=False)
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([np.outer(st, np.cos(phis)).ravel(), np.outer(st, np.sin(phis)).ravel(),
                     np.repeat(ct, phis.size)], 1)
    w = np.repeat(wt, phis.size) * (2 * np.pi / phis.size)
    Y, _ = oracle.sh_basis(3, dirs)
    gram = (Y * w[:, None]).T @ Y
    assert np.abs(gram - np.eye(16)).max() < 1e-12
    rng = np.random.default_rng(1)
    d = rng.normal(size=(20, 3))
    _, dY = oracle.sh_basis(3, d)
    h = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        Yp, _ = oracle.sh_basis(3, d + e)
        Ym, _ = oracle.sh_basis(3, d - e)
        assert np.abs((Yp - Ym) / (2 * h) - dY[:, :, a]).max() < 1e-7


# --------------------------------------------------------------------------
# Forward colour: closed forms (Section 3, Eq. alpha_blend / sigma_2D)
# --------------------------------------------------------------------------

def test_single_opaque_gaussian_centre_pixel():
    """o -> 0.999 on the optical axis: alpha is clamped at 0.99, so the centre
    pixel is exactly 0.99 c + 0.01 bg."""
    c0 = 0.5 / SQRT_PI
    dc = np.array([0.6, -0.4, 0.0]) / c0      # colour c = 0.5 + c0 dc
    colour = 0.5 + c0 * dc.astype(np.float32).astype(np.float64)
    sc = _one_gaussian([0, 0, 3.0], [-3.0, -3.0, -3.0], math.log(0.999 / 0.001), dc)
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings(bg=(0.2, 0.3, 0.4))
    r = oracle.render(sc, cam, st)
    a = float(np.float32(0.99))
    expect = a * colour + (1 - a) * np.array(st.bg, dtype=np.float32).astype(np.float64)
    assert np.abs(r["image"][32, 32] - expect).max() < 1e-12
    assert r["n_contrib"][32, 32] == 1


def test_single_gaussian_off_centre_closed_form():
    """Axis-aligned Gaussian on the optical axis: J is diagonal, so
    Sigma2D = diag(fx^2 sx^2/z^2 + 0.3, fy^2 sy^2/z^2 + 0.3) and
    C(x) = c o exp(-dx^2/(2 sx'^2) - dy^2/(2 sy'^2)) where composited."""
    sx, sy, z, o = 0.05, 0.03, 3.0, 0.5
    sc = _one_gaussian([0, 0, z], [math.log(sx), math.log(sy), -3.0], 0.0, [0.0, 0.0, 0.0])
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings()
    r = oracle.render(sc, cam, st)
    fx = 64.0
    s32x = math.exp(float(np.float32(math.log(sx))))   # the stored log-scale is float32
    s32y = math.exp(float(np.float32(math.log(sy))))
    vx = fx * fx * s32x ** 2 / z ** 2 + float(np.float32(0.3))
    vy = fx * fx * s32y ** 2 / z ** 2 + float(np.float32(0.3))
    checked = 0
    for py in range(26, 39):
        for px in range(26, 39):
            dx, dy = px - 32.0, py - 32.0
            a = o * math.exp(-0.5 * (dx * dx / vx + dy * dy / vy))
            if a < 1 / 255 * 1.001:
                continue
            assert abs(r["image"][py, px, 0] - 0.5 * a) < 1e-12
            checked += 1
    assert checked > 20


def test_two_gaussians_composite_by_hand():
    """Two Gaussians at distinct depths on the axis: C = c1 a1 + c2 a2 (1 - a1)
    + bg (1 - a1)(1 - a2) at the centre, whatever their input order."""
    c0 = 0.5 / SQRT_PI
    cols = np.array([[0.9, 0.2, 0.1], [0.1, 0.7, 0.4]])
    dcs = (cols - 0.5) / c0
    for order in ([0, 1], [1, 0]):
        means = np.array([[0, 0, 2.0], [0, 0, 3.5]])[order]
        logits = np.array([0.3, -0.2])[order]
        sc = _one_gaussian(means, [[-3.0] * 3] * 2, logits, dcs[order])
        cam = synth.camera_identity(64, 64, 64.0)
        st = synth.Settings(bg=(0.25, 0.5, 0.75))
        r = oracle.render(sc, cam, st)
        o = 1 / (1 + np.exp(-np.array([0.3, -0.2], dtype=np.float32).astype(np.float64)))
        bg = np.array(st.bg, dtype=np.float32).astype(np.float64)
        cc = 0.5 + c0 * dcs.astype(np.float32).astype(np.float64)
        expect = cc[0] * o[0] + cc[1] * o[1] * (1 - o[0]) + bg * (1 - o[0]) * (1 - o[1])
        assert np.abs(r["image"][32, 32] - expect).max() < 1e-12


def test_projection_against_pinhole_jacobian_and_library_rotation():
    """EWA projection by an independent route (Section 3, Eq. sigma_3D /
    sigma_2D): the 2-D mean is the pinhole map of R p + t, P its Jacobian
    with respect to p by central differences, Sigma_3D built with SciPy's
    quaternion rotation, Sigma_2D = P Sigma_3D P^T + 0.3 I and the conic its
    inverse; opacity is the logistic of the logit."""
    from scipy.spatial.transform import Rotation
    sc = synth.cluster_scene(4, 400, 0)
    cam = synth.camera_lookat((0.5, -0.3, -6.0), (0, 0, 0), 160, 120, 160.0)
    st = synth.Settings()
    pr = oracle.project(sc, cam, st)
    R = cam.R.astype(np.float64)
    t = cam.t.astype(np.float64)

    def pix(p):
        x, y, z = R @ p + t
        return np.array([cam.fx * x / z + cam.cx, cam.fy * y / z + cam.cy])

    lim_x, lim_y = 1.3 * 0.5 * cam.width / cam.fx, 1.3 * 0.5 * cam.height / cam.fy
    checked = 0
    for i in range(sc.n):
        p = sc.means[i].astype(np.float64)
        x, y, z = R @ p + t
        if pr["tiles"][i] == 0 or abs(x / z) >= lim_x or abs(y / z) >= lim_y:
            continue                                   # culled, or the Jacobian clamp is active
        checked += 1
        assert np.allclose(pr["mean2d"][i], pix(p), rtol=0, atol=1e-9)
        assert abs(pr["depth"][i] - z) < 1e-12
        h = 1e-5
        P = np.stack([(pix(p + h * e) - pix(p - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        assert np.allclose(pr["P"][i], P, rtol=1e-7, atol=1e-7 * np.abs(P).max())
        w, qx, qy, qz = sc.quats[i].astype(np.float64)
        Rq = Rotation.from_quat([qx, qy, qz, w]).as_matrix()           # SciPy: scalar last
        S3 = Rq @ np.diag(np.exp(2.0 * sc.log_scales[i].astype(np.float64))) @ Rq.T
        S2 = pr["P"][i] @ S3 @ pr["P"][i].T + float(np.float32(st.dilation)) * np.eye(2)   # settings are float32
        Q = np.linalg.inv(S2)
        assert np.allclose(pr["conic"][i], [Q[0, 0], Q[0, 1], Q[1, 1]], rtol=1e-9, atol=0)
        o = 1.0 / (1.0 + math.exp(-float(sc.opacity_logit[i])))
        assert abs(pr["opacity"][i] - o) < 1e-12
    assert checked > 100


# --------------------------------------------------------------------------
# Integer stages: brute force (binning, sort, ranges, rect coverage)
# --------------------------------------------------------------------------

def _brute_bins(scene, cam, st):
    isg = oracle.integer_stage(scene, cam, st)
    gx, gy = oracle.n_tiles(cam, st)
    inst = []
    for i in range(scene.n):
        if isg["tiles"][i] == 0:
            continue
        xl, xh, yl, yh = isg["rect"][i]
        db = int(isg["depth"][i:i + 1].view(np.uint32)[0])
        for ty in range(gy):
            for tx in range(gx):
                if xl <= tx <= xh and yl <= ty <= yh:
                    inst.append((ty * gx + tx, db, i))
    inst.sort()
    return isg, inst, gx * gy


@pytest.mark.parametrize("seed", [0, 5, 11])
def test_binning_sort_ranges_brute_force(seed):
    sc = synth.tiny_scene(seed)
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings()
    keys, gids, ranges = oracle.bin_sort(sc, cam, st)
    isg, inst, T = _brute_bins(sc, cam, st)
    assert len(inst) == len(keys) == int(isg["tiles"].sum())
    assert [t for t, _, _ in inst] == [int(k >> np.uint64(32)) for k in keys]
    assert [d for _, d, _ in inst] == [int(k & np.uint64(0xFFFFFFFF)) for k in keys]
    assert [g for _, _, g in inst] == gids.tolist()
    for t in range(T):
        idx = [k for k, x in enumerate(inst) if x[0] == t]
        if idx:
            assert ranges[t].tolist() == [idx[0], idx[-1] + 1]
        else:
            assert ranges[t, 0] == ranges[t, 1]


def test_rect_covers_three_sigma_ellipse_and_is_tight():
    """Every pixel within radius_sigma Mahalanobis distance of a visible
    Gaussian lies in a tile of its rect; every tile of the rect meets the
    square [mu - r, mu + r]."""
    sc = synth.tiny_scene(3)
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings()
    isg = oracle.integer_stage(sc, cam, st)
    pr = oracle.project(sc, cam, st)
    ys, xs = np.mgrid[0:64, 0:64]
    for i in range(sc.n):
        if isg["tiles"][i] == 0:
            continue
        q = pr["conic"][i]
        dx, dy = xs - pr["mean2d"][i, 0], ys - pr["mean2d"][i, 1]
        maha = q[0] * dx * dx + 2 * q[1] * dx * dy + q[2] * dy * dy
        inside = maha <= st.radius_sigma ** 2 * (1 - 1e-6)
        xl, xh, yl, yh = isg["rect"][i]
        tx, ty = xs // st.tile_w, ys // st.tile_h
        in_rect = (tx >= xl) & (tx <= xh) & (ty >= yl) & (ty <= yh)
        assert not np.any(inside & ~in_rect)
        # tightness: the rect is the set of tiles meeting the bounding square
        Sig = np.linalg.inv(np.array([[q[0], q[1]], [q[1], q[2]]]))
        m, det = 0.5 * (Sig[0, 0] + Sig[1, 1]), np.linalg.det(Sig)
        r = math.ceil(st.radius_sigma * math.sqrt(m + math.sqrt(max(0.1, m * m - det))))
        mx, my = isg["mean2d"][i]
        assert xl == max(0, math.floor((mx - r) / 16)) and xh == min(3, math.floor((mx + r) / 16))
        assert yl == max(0, math.floor((my - r) / 16)) and yh == min(3, math.floor((my + r) / 16))


def test_equal_depths_sort_by_gaussian_index():
    """Copies of one Gaussian share tiles and depth bits; within a tile they
    follow each other in increasing index (the stable order over instances
    emitted in index order), between the neighbours of their depth."""
    sc = synth.tiny_scene(2, 60)
    for i in (41, 7, 23):                            # copies of Gaussian 12, placed at shuffled indices
        for f in ("means", "log_scales", "quats", "opacity_logit", "sh"):
            getattr(sc, f)[i] = getattr(sc, f)[12]
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings()
    isg = oracle.integer_stage(sc, cam, st)
    assert isg["tiles"][12] > 0
    keys, gids, ranges = oracle.bin_sort(sc, cam, st)
    copies = [7, 12, 23, 41]
    for t in range(len(ranges)):
        a, b = ranges[t]
        g = gids[a:b].tolist()
        if 12 not in g:
            continue
        pos = [g.index(c) for c in copies]
        assert pos == list(range(pos[0], pos[0] + 4))   # adjacent, in index order
        d = [int(k & np.uint64(0xFFFFFFFF)) for k in keys[a:b]]
        assert d == sorted(d)


def test_near_plane_culls_and_renders_nothing():
    """A Gaussian whose camera depth is at or in front of the near plane
    (t_z <= 0.2) touches no tile and leaves the background; just behind it
    the same Gaussian is binned and drawn."""
    st = synth.Settings(bg=(0.1, 0.2, 0.3))
    cam = synth.camera_identity(64, 64, 64.0)
    near = np.float32(cam.near_z)
    for z, visible in ((0.15, False), (float(near), False), (float(np.nextafter(near, np.float32(1))), True),
                       (0.5, True)):
        sc = _one_gaussian([0.0, 0.0, z], [-3.0] * 3, 2.0, [1.0, 1.0, 1.0])
        isg = oracle.integer_stage(sc, cam, st)
        img = oracle.render(sc, cam, st)["image"]
        keys, _, _ = oracle.bin_sort(sc, cam, st)
        if visible:
            assert isg["tiles"][0] > 0 and len(keys) == isg["tiles"][0]
            assert np.abs(img - np.array(st.bg)).max() > 1e-3
        else:
            assert isg["tiles"][0] == 0 and len(keys) == 0
            bg = np.array(st.bg, np.float32).astype(np.float64)     # the settings carry float32
            assert np.array_equal(img, np.broadcast_to(bg, img.shape))


# --------------------------------------------------------------------------
# Gradients: central finite differences on the full model (smooth mode)
# --------------------------------------------------------------------------

FIELDS = ("means", "log_scales", "quats", "opacity_logit", "sh")


def _lin_loss(scene, cam, st, g):
    return float(np.sum(oracle.render(scene, cam, st)["image"] * g))


def _fd_check(scene, cam, st, g, gauss_idx, h=1e-4):
    ana = oracle.backward(scene, cam, st, g)
    base_keys = oracle.bin_sort(scene, cam, st)[1]
    fd_all, an_all = [], []
    for i in gauss_idx:
        for f in FIELDS:
            arr = getattr(scene, f)
            flat = arr.reshape(scene.n, -1)
            for k in range(flat.shape[1]):
                x0 = flat[i, k]
                vals = []
                ok = True
                for s in (+1, -1):
                    sc2 = scene.copy()
                    a2 = getattr(sc2, f).reshape(scene.n, -1)
                    a2[i, k] = np.float32(x0 + s * h)
                    if not np.array_equal(oracle.bin_sort(sc2, cam, st)[1], base_keys):
                        ok = False
                        break
                    vals.append((_lin_loss(sc2, cam, st, g), float(a2[i, k])))
                if not ok:
                    continue
                (lp, xp), (lm, xm) = vals
                fd_all.append((lp - lm) / (xp - xm))
                an_all.append(ana[f if f != "opacity_logit" else "opacity_logit"].reshape(scene.n, -1)[i, k])
    return np.array(fd_all), np.array(an_all)


def test_gradient_matches_central_differences_sh0():
    sc = synth.tiny_scene(0)
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings().smooth()
    g = np.random.default_rng(7).normal(size=(64, 64, 3)) / (64 * 64)
    vis = np.nonzero(oracle.integer_stage(sc, cam, st)["tiles"])[0]
    idx = np.random.default_rng(3).choice(vis, 16, replace=False)
    fd, an = _fd_check(sc, cam, st, g, idx)
    assert fd.size > 150
    err = np.linalg.norm(fd - an) / np.linalg.norm(an)
    assert err < 1e-5, err
    assert np.abs(fd - an).max() < 1e-4 * np.abs(an).max()


def test_gradient_matches_central_differences_sh3_offaxis():
    """Degree-3 SH (view-dependent colour depends on p) and an off-axis,
    rotated camera with Gaussians near the Jacobian clamp."""
    sc = synth.cluster_scene(4, 96, sh_degree=3)
    sc.log_scales[:] = sc.log_scales + 2.0          # a few pixels wide at this distance
    cam = synth.camera_lookat((1.0, -0.5, -6.0), (0.3, 0.2, 0.0), 48, 40, 48.0)
    st = synth.Settings().smooth()
    st.fov_clamp = 1.05
    g = np.random.default_rng(8).normal(size=(40, 48, 3)) / (48 * 40)
    vis = np.nonzero(oracle.integer_stage(sc, cam, st)["tiles"])[0]
    idx = np.random.default_rng(4).choice(vis, min(6, vis.size), replace=False)
    fd, an = _fd_check(sc, cam, st, g, idx)
    assert fd.size > 200
    err = np.linalg.norm(fd - an) / np.linalg.norm(an)
    assert err < 1e-5, err


def test_gradient_with_active_alpha_clamp():
    """Where o G > alpha_max the composited alpha is the constant alpha_max: its
    derivative is zero, which central differences confirm away from the kink."""
    sc = synth.tiny_scene(2, 32)
    sc.opacity_logit[:] = 6.0                      # o ~ 0.9975: clamp active near centres
    cam = synth.camera_identity(32, 32, 32.0)
    st = synth.Settings().smooth()
    st.alpha_max = 0.99
    g = np.random.default_rng(9).normal(size=(32, 32, 3)) / (32 * 32)
    vis = np.nonzero(oracle.integer_stage(sc, cam, st)["tiles"])[0]
    fd, an = _fd_check(sc, cam, st, g, vis[:8], h=1e-4)
    err = np.linalg.norm(fd - an) / np.linalg.norm(an)
    assert err < 1e-3, err


def test_l1_loss_gradient():
    rng = np.random.default_rng(0)
    img = rng.uniform(size=(8, 9, 3))
    tgt = rng.uniform(size=(8, 9, 3)).astype(np.float32)
    L, g = oracle.l1_loss_grad(img, tgt, n_views=2)
    assert abs(L - np.mean(np.abs(img - tgt.astype(np.float64))) / 2) < 1e-15
    h = 1e-7
    for k in range(10):
        idx = tuple(rng.integers(0, s) for s in img.shape)
        e = np.zeros_like(img)
        e[idx] = h
        fd = (oracle.l1_loss_grad(img + e, tgt, 2)[0] - oracle.l1_loss_grad(img - e, tgt, 2)[0]) / (2 * h)
        assert abs(fd - g[idx]) < 1e-9


# --------------------------------------------------------------------------
# Splitting matrix = Hessian of the loss w.r.t. p_i in the frozen model
# (Theorem 1 with T^(i) = 0 for a loss affine in each alpha, Lemma on the
# decomposition of the Hessian, and the Appendix's closed-form Hessian).
# --------------------------------------------------------------------------

def _frozen_hessian(sc, cam, st, i, g, h):
    H = np.zeros((3, 3))
    f0 = oracle.frozen_eval(sc, cam, st, i, dp=np.zeros(3), g=g)
    for a in range(3):
        for b in range(a, 3):
            def f(sa, sb):
                d = np.zeros(3)
                d[a] += sa * h
                d[b] += sb * h
                return oracle.frozen_eval(sc, cam, st, i, dp=d, g=g)
            if a == b:
                v = (f(1, 0) - 2 * f0 + f(-1, 0)) / h ** 2
            else:
                v = (f(1, 1) - f(1, -1) - f(-1, 1) + f(-1, -1)) / (4 * h * h)
            H[a, b] = H[b, a] = v
    return H


def test_splitting_matrix_equals_frozen_hessian():
    sc = synth.tiny_scene(0)
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings().smooth()
    g = np.random.default_rng(11).normal(size=(64, 64, 3)) / (64 * 64)
    S = oracle.backward(sc, cam, st, g)["S"]
    vis = np.nonzero(oracle.integer_stage(sc, cam, st)["tiles"])[0]
    for i in np.random.default_rng(5).choice(vis, 8, replace=False):
        # Richardson: H(h) = H + c h^2 + ..., so (4 H(h/2) - H(h)) / 3 = H + O(h^4)
        h = 2e-3
        H1 = _frozen_hessian(sc, cam, st, i, g, h)
        H2 = _frozen_hessian(sc, cam, st, i, g, h / 2)
        Hr = (4 * H2 - H1) / 3
        rel = np.linalg.norm(Hr - S[i]) / np.linalg.norm(S[i])
        assert rel < 1e-6, (i, rel)


def test_splitting_matrix_symmetric():
    sc = synth.tiny_scene(1)
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings()
    r = oracle.render(sc, cam, st)
    _, g = oracle.l1_loss_grad(r["image"], synth.target_image(2, 64, 64))
    S = oracle.backward(sc, cam, st, g)["S"]
    assert np.array_equal(S, np.transpose(S, (0, 2, 1)))
    assert np.abs(S).max() > 0


# --------------------------------------------------------------------------
# Theorems 1 and 2: sign of lambda_min decides; predicted decrease; optimality
# --------------------------------------------------------------------------

def _setup_l1(seed=0):
    sc = synth.tiny_scene(seed)
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings().smooth()
    r = oracle.render(sc, cam, st)
    tgt = synth.target_image(2, 64, 64)
    _, g = oracle.l1_loss_grad(r["image"], tgt)
    S = oracle.backward(sc, cam, st, g)["S"]
    return sc, cam, st, g, tgt, S


def test_split_sign_and_predicted_decrease():
    """Mixture split of Gaussian i along +-eps v (w = 1/2):
    L(split) - L(theta) = eps^2 v^T S v / 2 + O(eps^4); with v = v_min the change
    is negative iff lambda_min < 0.  Checked on the linear functional (exact
    second order) and on the real L1 loss."""
    sc, cam, st, g, tgt, S = _setup_l1(0)
    lam, v = oracle.eig3_min(S)
    ev, V = oracle.jacobi3(S)
    base_lin = oracle.frozen_eval(sc, cam, st, 0, dp=np.zeros(3), g=g)
    base_l1 = oracle.frozen_eval(sc, cam, st, 0, dp=np.zeros(3), target=tgt)
    scale = np.abs(S).reshape(len(S), -1).max(1)
    cand = [i for i in np.argsort(-scale)[:12]]
    n_neg = n_pos = 0
    for i in cand:
        s_max = float(np.exp(sc.log_scales[i].astype(np.float64)).max())
        errs = []
        for frac in (1e-1, 3e-2, 1e-2):
            eps = frac * s_max
            pred = 0.5 * eps * eps * lam[i]
            meas = oracle.frozen_eval(sc, cam, st, i, mix_v=eps * v[i], g=g) - base_lin
            errs.append(abs(meas - pred))
            if frac == 1e-2:
                assert abs(meas - pred) <= 1e-3 * abs(pred) + 1e-15
                assert (meas < 0) == (lam[i] < 0)
                meas1 = oracle.frozen_eval(sc, cam, st, i, mix_v=eps * v[i], target=tgt) - base_l1
                assert (meas1 < 0) == (lam[i] < 0)
                # the largest eigenvector direction gives the largest eigenvalue's change
                pmax = 0.5 * eps * eps * ev[i, 2]
                mmax = oracle.frozen_eval(sc, cam, st, i, mix_v=eps * V[i, 2], g=g) - base_lin
                assert abs(mmax - pmax) <= 1e-3 * abs(pmax) + 1e-15
        # remainder is higher order (symmetric split => odd orders cancel)
        slope = np.log(errs[0] / errs[2]) / np.log(10.0)
        assert slope > 2.9, slope
        n_neg += lam[i] < 0
        n_pos += ev[i, 2] > 0
    assert n_neg > 0 and n_pos > 0


def test_split_along_v_min_is_optimal():
    """No direction beats +-v_min (Theorem 2): over random unit directions the
    second-order change never goes below eps^2 lambda_min / 2."""
    sc, cam, st, g, tgt, S = _setup_l1(1)
    lam, v = oracle.eig3_min(S)
    i = int(np.argmin(lam))
    eps = 1e-2 * float(np.exp(sc.log_scales[i].astype(np.float64)).max())
    base = oracle.frozen_eval(sc, cam, st, i, dp=np.zeros(3), g=g)
    best = oracle.frozen_eval(sc, cam, st, i, mix_v=eps * v[i], g=g) - base
    rng = np.random.default_rng(0)
    for _ in range(300):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        dv = oracle.frozen_eval(sc, cam, st, i, mix_v=eps * d, g=g) - base
        assert dv >= best - 1e-6 * abs(best)


# --------------------------------------------------------------------------
# Eigen-solve: trig formula vs Jacobi vs LAPACK, identities, degenerate cases
# --------------------------------------------------------------------------

def _rand_sym(rng, n):
    A = rng.normal(size=(n, 3, 3))
    return A + np.transpose(A, (0, 2, 1))


def test_eig_trig_matches_jacobi_and_lapack():
    rng = np.random.default_rng(0)
    A = _rand_sym(rng, 2000)
    # known spectra: U diag(l) U^T with repeated and near-repeated eigenvalues
    U = np.linalg.qr(rng.normal(size=(300, 3, 3)))[0]
    ls = rng.normal(size=(300, 3))
    ls[:100, 1] = ls[:100, 0]
    ls[100:150, 1] = ls[100:150, 0] + 1e-9
    B = np.einsum("nij,nj,nkj->nik", U, ls, U)
    A = np.concatenate([A, B])
    lam, v = oracle.eig3_min(A)
    ev, V = oracle.jacobi3(A)
    ref = np.linalg.eigvalsh(A)
    nrm = np.linalg.norm(A.reshape(len(A), -1), axis=1)
    sep = (ref[:, 1] - ref[:, 0]) > 1e-6 * nrm
    # arccos near +-1 loses half the digits at a repeated minimum eigenvalue
    assert np.all(np.abs(lam - ref[:, 0])[sep] <= 1e-12 * nrm[sep])
    assert np.all(np.abs(lam - ref[:, 0]) <= 1e-7 * nrm)
    assert np.all(np.abs(ev - ref) <= 1e-12 * nrm[:, None])
    res = np.linalg.norm(np.einsum("nij,nj->ni", A, v) - lam[:, None] * v, axis=1)
    gap = ref[:, 1] - ref[:, 0]
    ok = gap > 1e-6 * nrm
    assert np.all(res[ok] <= 1e-10 * nrm[ok])
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-14)
    # trace and determinant identities (Jacobi's full spectrum)
    assert np.all(np.abs(ev.sum(1) - np.trace(A, axis1=1, axis2=2)) <= 1e-12 * nrm)
    assert np.all(np.abs(ev.prod(1) - np.linalg.det(A)) <= 1e-11 * nrm ** 3)
    # agreement of eigenvectors where the gap is clear
    cosang = np.abs(np.einsum("ni,ni->n", v, V[:, 0, :]))
    assert np.all(1 - cosang[ok & (gap > 1e-3 * nrm)] < 1e-10)


def test_eig_degenerate_cases():
    # zero and scalar matrices: lambda = q, v = e_x
    lam, v = oracle.eig3_min(np.stack([np.zeros((3, 3)), 2.5 * np.eye(3)]))
    assert lam.tolist() == [0.0, 2.5]
    assert v.tolist() == [[1, 0, 0], [1, 0, 0]]
    # diagonal: exact minimum and axis
    lam, v = oracle.eig3_min(np.diag([3.0, -1.0, 2.0])[None])
    assert abs(lam[0] + 1.0) < 1e-14 and np.allclose(v[0], [0, 1, 0], atol=1e-12)
    # rank-one negative: double zero eigenvalue above a negative one
    u = np.array([1.0, 2.0, -2.0]) / 3.0
    lam, v = oracle.eig3_min((-4.0 * np.outer(u, u))[None])
    assert abs(lam[0] + 4.0) < 1e-12 and abs(abs(v[0] @ u) - 1) < 1e-12
    # repeated minimum: v is any unit vector of the eigenspace, canonical sign
    lam, v = oracle.eig3_min(np.diag([-1.0, -1.0, 5.0])[None])
    assert abs(lam[0] + 1.0) < 1e-12 and abs(v[0, 2]) < 1e-12
    assert abs(np.linalg.norm(v[0]) - 1) < 1e-12
    k = int(np.argmax(np.abs(v[0])))
    assert v[0, k] > 0


# --------------------------------------------------------------------------
# Split output (Theorem 2, Algorithm 1)
# --------------------------------------------------------------------------

def test_split_output_invariants():
    sc, cam, st, g, tgt, S = _setup_l1(0)
    lam, v = oracle.eig3_min(S)
    out = oracle.split(sc, lam, v, eps_split=-1e-6, step_scale=0.5)
    flags = lam < -1e-6
    n = sc.n
    assert out["n_out"] == n + flags.sum()
    assert np.array_equal(out["flags"], flags)
    par = out["parent"]
    assert np.array_equal(par[:n], np.arange(n))
    assert np.array_equal(par[n:], np.nonzero(flags)[0])
    o = 1 / (1 + np.exp(-sc.opacity_logit.astype(np.float64)))
    for row2, i in enumerate(np.nonzero(flags)[0]):
        j = n + row2
        m1, m2 = out["means"][i], out["means"][j]
        assert np.allclose(0.5 * (m1 + m2), sc.means[i].astype(np.float64), atol=1e-12)
        eps = 0.5 * np.exp(sc.log_scales[i].astype(np.float64)).max()
        assert np.allclose(m1 - m2, 2 * eps * v[i], atol=1e-12)
        o1 = 1 / (1 + np.exp(-out["opacity_logit"][i]))
        o2 = 1 / (1 + np.exp(-out["opacity_logit"][j]))
        assert abs(o1 + o2 - o[i]) < 1e-12 and abs(o1 - o2) < 1e-15
        for f in ("log_scales", "quats", "sh"):
            assert np.array_equal(out[f][j], getattr(sc, f)[i].astype(np.float64))
    keep = ~flags
    assert np.array_equal(out["means"][:n][keep], sc.means[keep].astype(np.float64))
    assert np.array_equal(out["opacity_logit"][:n][keep], sc.opacity_logit[keep].astype(np.float64))
    # gradient gate (compactest condition)
    gn = np.random.default_rng(0).uniform(size=n)
    out2 = oracle.split(sc, lam, v, -1e-6, 0.5, grad_norm=gn, eps_grad=0.5)
    assert np.array_equal(out2["flags"], flags & (gn <= 0.5))


def test_split_with_given_flags_is_the_scan_of_those_flags():
    """The split driven by a given flag vector (how GPU decisions are handed
    to the oracle's scan): with the rule's own flags it reproduces the rule's
    output exactly; with arbitrary flags the appended rows are the flagged
    indices in increasing order (the exclusive scan), each pair sits
    symmetrically about its parent at distance eps_i along v, and unflagged
    rows are copied."""
    sc, cam, st, g, tgt, S = _setup_l1(0)
    lam, v = oracle.eig3_min(S)
    n = sc.n
    rule = oracle.split(sc, lam, v, eps_split=-1e-6, step_scale=0.5)
    same = oracle.split(sc, lam, v, eps_split=-1e-6, step_scale=0.5, flags=rule["flags"])
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh", "parent", "flags"):
        assert np.array_equal(same[k], rule[k]), k
    rng = np.random.default_rng(9)
    for p_flag in (0.0, 0.3, 1.0):
        f = rng.uniform(size=n) < p_flag
        out = oracle.split(sc, lam, v, eps_split=-1e-6, step_scale=0.5, flags=f)
        assert out["n_out"] == n + f.sum() and np.array_equal(out["flags"], f)
        par = out["parent"]
        assert np.array_equal(par[:n], np.arange(n))
        assert list(par[n:]) == [i for i in range(n) if f[i]]
        for r, i in enumerate(np.nonzero(f)[0]):
            j = n + r
            eps = 0.5 * np.exp(sc.log_scales[i].astype(np.float64)).max()
            np.testing.assert_allclose(out["means"][i] - out["means"][j], 2 * eps * v[i], atol=1e-12)
            np.testing.assert_allclose(out["means"][i] + out["means"][j], 2 * sc.means[i].astype(np.float64),
                                       atol=1e-12)
        keep = ~f
        assert np.array_equal(out["means"][:n][keep], sc.means[keep].astype(np.float64))
        assert np.array_equal(out["opacity_logit"][:n][keep], sc.opacity_logit[keep].astype(np.float64))
    # the (p, o) split takes given flags the same way
    acc = oracle.backward(sc, cam, st, g)
    lam4, v4 = oracle.eig_min_sym(oracle.S4_matrix(acc["S"], acc["S_po"]))
    r4 = oracle.split_po(sc, lam4, v4, -1e-9, 0.5)
    s4 = oracle.split_po(sc, lam4, v4, -1e-9, 0.5, flags=r4["flags"])
    for k in ("means", "opacity_logit", "parent", "flags"):
        assert np.array_equal(s4[k], r4[k]), k
    f = rng.uniform(size=n) < 0.4
    o4 = oracle.split_po(sc, lam4, v4, -1e-9, 0.5, flags=f)
    assert list(o4["parent"][n:]) == [i for i in range(n) if f[i]]


def test_increment_budget_is_the_best_k_subset():
    """Increment budget (Appendix, "Densification with Increment Budget"): the
    second-order loss change of splitting Gaussian i along v_min is
    proportional to lambda_min(S_i), so among all admissible subsets of at
    most K candidates the chosen one has the least sum of lambda_min.  Brute
    force over every subset of a 9-Gaussian scene, with tied values and the
    gradient gate in play; among optimal subsets the lexicographically first
    by index."""
    import itertools
    sc = synth.tiny_scene(0)
    sc = synth.subset(sc, slice(0, 9))
    rng = np.random.default_rng(4)
    v = rng.normal(size=(9, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    lam = np.array([-3.0, 0.5, -1.0, -3.0, -2.0, -1.0, 0.0, -1.0, -4.0])
    gn = np.array([0.1, 0.1, 0.1, 0.1, 0.9, 0.1, 0.1, 0.1, 0.1])
    for eps_grad, gate in ((0.0, None), (0.5, gn)):
        base = oracle.split(sc, lam, v, 0.0, grad_norm=gate, eps_grad=eps_grad)["flags"]
        cand = np.nonzero(base)[0]
        for K in range(1, len(cand) + 2):
            got = oracle.split(sc, lam, v, 0.0, grad_norm=gate, eps_grad=eps_grad, budget=K)
            best = None
            for r in range(0, min(K, len(cand)) + 1):
                for sub in itertools.combinations(cand, r):
                    key = (lam[list(sub)].sum(), -len(sub), tuple(sub))
                    best = key if best is None or key < best else best
            want = np.zeros(9, bool)
            want[list(best[2])] = True
            assert np.array_equal(got["flags"], want), (eps_grad, K)
            assert got["n_out"] == 9 + want.sum()
            assert np.array_equal(got["parent"][9:], np.nonzero(want)[0])


# --------------------------------------------------------------------------
# Splitting matrices over theta = (p, o) (dim Theta = 4)
# --------------------------------------------------------------------------

def _frozen_mixed(sc, cam, st, i, g, h):
    """Central-difference d^2 (g.C) / dp_a do of the frozen model."""
    out = np.zeros(3)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        f = lambda dp, do: oracle.frozen_eval(sc, cam, st, i, dp=dp, d_o=do, g=g)   # noqa: E731
        out[a] = (f(e, h) - f(e, -h) - f(-e, h) + f(-e, -h)) / (4 * h * h)
    return out


def test_position_opacity_block_equals_frozen_hessian():
    sc = synth.tiny_scene(0)
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings().smooth()
    g = np.random.default_rng(11).normal(size=(64, 64, 3)) / (64 * 64)
    acc = oracle.backward(sc, cam, st, g)
    vis = np.nonzero(oracle.integer_stage(sc, cam, st)["tiles"])[0]
    for i in np.random.default_rng(6).choice(vis, 6, replace=False):
        h = 2e-3
        Hr = (4 * _frozen_mixed(sc, cam, st, i, g, h / 2) - _frozen_mixed(sc, cam, st, i, g, h)) / 3
        rel = np.linalg.norm(Hr - acc["S_po"][i]) / np.linalg.norm(acc["S_po"][i])
        assert rel < 1e-6, (i, rel)
        # sigma is linear in o: the opacity-opacity entry is zero
        f0 = oracle.frozen_eval(sc, cam, st, i, dp=np.zeros(3), g=g)
        fp = oracle.frozen_eval(sc, cam, st, i, dp=np.zeros(3), d_o=0.05, g=g)
        fm = oracle.frozen_eval(sc, cam, st, i, dp=np.zeros(3), d_o=-0.05, g=g)
        assert abs(fp - 2 * f0 + fm) <= 1e-12 * (abs(fp) + abs(fm))


def test_4d_split_predicted_decrease_interlacing_and_optimality():
    sc, cam, st, g, tgt, S = _setup_l1(0)
    acc = oracle.backward(sc, cam, st, g)
    S4 = oracle.S4_matrix(acc["S"], acc["S_po"])
    lam4, v4 = oracle.eig_min_sym(S4)
    lam3 = np.linalg.eigvalsh(acc["S"])[:, 0]
    # adding the opacity row and column can only lower the minimum (interlacing)
    assert np.all(lam4 <= np.minimum(lam3, 0.0) + 1e-12 * np.abs(S4).reshape(len(S4), -1).max(1))
    # block-diagonal special case: no mixed block -> min(lambda_min(S_pp), 0)
    l0, _ = oracle.eig_min_sym(oracle.S4_matrix(acc["S"], np.zeros_like(acc["S_po"])))
    np.testing.assert_allclose(l0, np.minimum(lam3, 0.0), rtol=0, atol=1e-12 * np.abs(acc["S"]).max())
    base = oracle.frozen_eval(sc, cam, st, 0, dp=np.zeros(3), g=g)
    scale = np.abs(S4).reshape(len(S4), -1).max(1)
    for i in np.argsort(-scale)[:6]:
        s_max = float(np.exp(sc.log_scales[i].astype(np.float64)).max())
        eps = 1e-2 * s_max
        pred = 0.5 * eps * eps * lam4[i]
        meas = oracle.frozen_eval(sc, cam, st, i, mix_v=eps * v4[i, :3], d_o=eps * v4[i, 3], g=g) - base
        assert abs(meas - pred) <= 1e-3 * abs(pred) + 1e-15, (i, meas, pred)
        rng = np.random.default_rng(int(i))
        for _ in range(60):
            d = rng.normal(size=4)
            d /= np.linalg.norm(d)
            dv = oracle.frozen_eval(sc, cam, st, i, mix_v=eps * d[:3], d_o=eps * d[3], g=g) - base
            assert dv >= meas - 1e-3 * abs(meas) - 1e-15


def test_split_po_output_invariants():
    sc, cam, st, g, tgt, S = _setup_l1(0)
    acc = oracle.backward(sc, cam, st, g)
    lam4, v4 = oracle.eig_min_sym(oracle.S4_matrix(acc["S"], acc["S_po"]))
    out = oracle.split_po(sc, lam4, v4, eps_split=-1e-9, step_scale=0.5)
    flags = lam4 < -1e-9
    n = sc.n
    assert out["n_out"] == n + flags.sum() and np.array_equal(out["flags"], flags)
    assert np.array_equal(out["parent"][n:], np.nonzero(flags)[0])
    o = 1 / (1 + np.exp(-sc.opacity_logit.astype(np.float64)))
    for r, i in enumerate(np.nonzero(flags)[0]):
        j = n + r
        eps = 0.5 * np.exp(sc.log_scales[i].astype(np.float64)).max()
        np.testing.assert_allclose(out["means"][i] - out["means"][j], 2 * eps * v4[i, :3], atol=1e-12)
        o1 = 1 / (1 + np.exp(-out["opacity_logit"][i]))
        o2 = 1 / (1 + np.exp(-out["opacity_logit"][j]))
        want1 = np.clip(0.5 * (o[i] + eps * v4[i, 3]), 1e-4, 1 - 1e-4)
        want2 = np.clip(0.5 * (o[i] - eps * v4[i, 3]), 1e-4, 1 - 1e-4)
        assert abs(o1 - want1) < 1e-12 and abs(o2 - want2) < 1e-12
        if want1 > 1e-4 and want2 > 1e-4:
            assert abs(o1 + o2 - o[i]) < 1e-12
    keep = ~flags
    assert np.array_equal(out["means"][:n][keep], sc.means[keep].astype(np.float64))


# --------------------------------------------------------------------------
# Splitting matrices over theta = (p, l, o), l the log-scales (dim Theta = 7)
# --------------------------------------------------------------------------

def _fz(sc, cam, st, i, g, dp=None, dls=None, do=0.0):
    return oracle.frozen_eval(sc, cam, st, i, dp=np.zeros(3) if dp is None else dp, d_ls=dls, d_o=do, g=g)


def _mixed(f, u, v, h):
    """Central-difference d^2 f / du dv for unit offsets u, v (callables of h)."""
    return (f(u(h), v(h)) - f(u(h), v(-h)) - f(u(-h), v(h)) + f(u(-h), v(-h))) / (4 * h * h)


def test_log_scale_blocks_equal_frozen_hessian():
    sc = synth.tiny_scene(0)
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings().smooth()
    g = np.random.default_rng(11).normal(size=(64, 64, 3)) / (64 * 64)
    acc = oracle.backward(sc, cam, st, g)
    S7 = oracle.S7_matrix(acc["S"], acc["S_po"], acc["S_ls"])
    vis = np.nonzero(oracle.integer_stage(sc, cam, st)["tiles"])[0]

    def e3(a, h):
        v = np.zeros(3)
        v[a] = h
        return v

    for i in np.random.default_rng(7).choice(vis, 4, replace=False):
        H = np.zeros((7, 7))
        for r in range(7):
            for c in range(r, 7):
                def f(x, y, r=r, c=c):
                    dp, dls, do = np.zeros(3), np.zeros(3), 0.0
                    for idx, val in ((r, x), (c, y)):
                        if idx < 3:
                            dp = dp + e3(idx, 1.0) * val
                        elif idx < 6:
                            dls = dls + e3(idx - 3, 1.0) * val
                        else:
                            do = do + val
                    return _fz(sc, cam, st, i, g, dp, dls, do)
                hr = []
                for h in (2e-3, 1e-3):
                    hr.append(_mixed(f, lambda t: t, lambda t: t, h) if r != c else
                              (f(h / 2, h / 2) - 2 * f(0.0, 0.0) + f(-h / 2, -h / 2)) / (h * h))
                H[r, c] = H[c, r] = (4 * hr[1] - hr[0]) / 3
        rel = np.linalg.norm(H - S7[i]) / np.linalg.norm(S7[i])
        assert rel < 1e-5, (i, rel)


def test_7d_split_predicted_decrease_interlacing_and_optimality():
    sc, cam, st, g, tgt, S = _setup_l1(0)
    acc = oracle.backward(sc, cam, st, g)
    S7 = oracle.S7_matrix(acc["S"], acc["S_po"], acc["S_ls"])
    lam7, v7 = oracle.eig_min_sym(S7)
    lam4, _ = oracle.eig_min_sym(oracle.S4_matrix(acc["S"], acc["S_po"]))
    scale = np.abs(S7).reshape(len(S7), -1).max(1)
    assert np.all(lam7 <= lam4 + 1e-12 * scale)
    base = oracle.frozen_eval(sc, cam, st, 0, dp=np.zeros(3), g=g)
    for i in np.argsort(-scale)[:5]:
        s_max = float(np.exp(sc.log_scales[i].astype(np.float64)).max())
        eps = 1e-2 * s_max
        v = v7[i]
        pred = 0.5 * eps * eps * lam7[i]
        meas = oracle.frozen_eval(sc, cam, st, i, mix_v=eps * v[:3], d_ls=eps * v[3:6], d_o=eps * v[6], g=g) - base
        assert abs(meas - pred) <= 1e-3 * abs(pred) + 1e-15, (i, meas, pred)
        rng = np.random.default_rng(int(i))
        for _ in range(40):
            d = rng.normal(size=7)
            d /= np.linalg.norm(d)
            dv = oracle.frozen_eval(sc, cam, st, i, mix_v=eps * d[:3], d_ls=eps * d[3:6], d_o=eps * d[6],
                                    g=g) - base
            assert dv >= meas - 1e-3 * abs(meas) - 1e-15
    out = oracle.split_po(sc, lam7, v7, eps_split=-1e-9, step_scale=0.5)
    n = sc.n
    for r, i in enumerate(np.nonzero(lam7 < -1e-9)[0][:20]):
        eps = 0.5 * np.exp(sc.log_scales[i].astype(np.float64)).max()
        np.testing.assert_allclose(out["log_scales"][i] - out["log_scales"][n + r], 2 * eps * v7[i, 3:6],
                                   atol=1e-12)


# --------------------------------------------------------------------------
# The all-core variants (a timing baseline) against the single-thread oracle
# --------------------------------------------------------------------------

def test_all_core_render_and_backward_equal_the_single_thread_oracle():
    sc = synth.cluster_scene(3, 3000, 3)
    cam = synth.camera_lookat((1.0, 0.5, -6.0), (0, 0, 0), 150, 101, 150.0)
    st = synth.Settings()
    r1 = oracle.render(sc, cam, st)
    rm = oracle.render(sc, cam, st, all_cores=True)
    for k in ("image", "final_T", "n_contrib", "band"):
        assert np.array_equal(r1[k], rm[k]), k
    _, g = oracle.l1_loss_grad(r1["image"], synth.target_image(2, cam.height, cam.width))
    a1 = oracle.backward(sc, cam, st, g)
    am = oracle.backward(sc, cam, st, g, all_cores=True)
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh", "S", "S_po", "S_ls", "grad2d"):
        d = np.linalg.norm(a1[k] - am[k]) / max(np.linalg.norm(a1[k]), 1e-300)
        assert d < 1e-12, (k, d)
    # a row window, and accumulation into an existing acc
    acc = oracle.backward(sc, cam, st, g[40:57], rows=(40, 17))
    accm = oracle.backward(sc, cam, st, g[40:57], rows=(40, 17), all_cores=True)
    assert np.linalg.norm(acc["S"] - accm["S"]) <= 1e-12 * np.linalg.norm(acc["S"])
