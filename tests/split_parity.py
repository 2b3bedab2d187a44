"""Split and compaction parity between the GPU's densify_split and the
oracle, with no branch on whether the two sides took the same decisions.

The GPU decides lambda_min < eps_split in float32, the oracle in float64, so
the two flag vectors may differ where lambda_min lies within rounding of the
threshold (the band).  The check therefore:

  1. reads the GPU's flags from its compaction (parent[n:] lists the split
     Gaussians) and requires parent[:n] = 0..n-1 and parent[n:] strictly
     increasing;
  2. requires the GPU flags to equal the oracle's rule outside the band, and
     the mismatches (all inside it) to number at most ceil(1e-4 n), not
     counting Gaussians whose lambda_min sits exactly at the threshold in
     exact arithmetic (`structural`: on one view S = P^T M P has rank <= 2,
     so lambda_min = 0 wherever M is positive semidefinite, and at
     eps_split = 0 both sides then decide on the sign of rounding error);
  3. hands the GPU's flags to the oracle's scan (Theorem 2, Algorithm 1:
     exclusive scan of the flags, the + offspring in the parent's row, the -
     offspring appended in index order) and compares every output row:
     n_out and parent bit for bit; copied attributes bit for bit; displaced
     means (and log-scales in the 7-D split) and opacities at the stated
     tolerances wherever the eigenvector is unique, and, where it is not, the
     pair's symmetry about its parent.
"""
import math

import numpy as np

import oracle


def gpu_flags(parent, n, n_out):
    """Split decisions recovered from the compaction: parent[n:n_out] are the
    split Gaussians, which must appear once each in increasing order."""
    par = np.asarray(parent[:n_out], np.int64)
    assert np.array_equal(par[:n], np.arange(n))
    tail = par[n:]
    assert np.all(np.diff(tail) > 0), "appended rows out of index order or repeated"
    assert tail.size == 0 or (tail[0] >= 0 and tail[-1] < n)
    f = np.zeros(n, bool)
    f[tail] = True
    return f


def structural_zeros(lam_exact, nrm_exact, eps_split, rel=1e-12):
    """Gaussians whose lambda_min, from the float64 oracle's own splitting
    matrices, equals eps_split up to float64 rounding: their decision is not
    determined by the method, only by rounding."""
    return np.abs(np.asarray(lam_exact) - eps_split) <= rel * np.maximum(np.asarray(nrm_exact), 1e-300)


def check_split(scene, out, parent, n_out, lam_o, v_o, flags_rule, decided, gap, eps_split, step_scale,
                dim=3, v_gpu=None, structural=None):
    """Compare the GPU split (output fields `out` as numpy arrays, `parent`,
    `n_out`) with the oracle's split of the GPU's own flags.

    lam_o, v_o: the oracle's eigenpairs; flags_rule: the oracle's decisions;
    decided: Gaussians outside the band (their decisions must agree);
    gap: Gaussians whose minimum eigenvector is unique (offspring positions
    compared there); v_gpu: the GPU's eigenvectors (a sign chosen differently
    on a near-tie of the two largest components swaps the offspring)."""
    n = scene.n
    flags_g = gpu_flags(parent, n, n_out)
    mism = flags_g != np.asarray(flags_rule, bool)
    assert not (mism & decided).any(), f"{int((mism & decided).sum())} split decisions differ outside the band"
    counted = mism if structural is None else mism & ~np.asarray(structural, bool)
    assert counted.sum() <= math.ceil(1e-4 * n), \
        f"{int(counted.sum())} banded decisions differ ({int(mism.sum())} with those at exactly the threshold)"
    if dim == 3:
        sp = oracle.split(scene, lam_o, v_o, eps_split, step_scale, flags=flags_g)
    else:
        sp = oracle.split_po(scene, lam_o, v_o, eps_split, step_scale, flags=flags_g)
    assert n_out == sp["n_out"]
    par = np.asarray(parent[:n_out], np.int64)
    assert np.array_equal(par, sp["parent"])
    copied = ("quats", "sh") if dim == 7 else ("log_scales", "quats", "sh")
    for f in copied:
        assert np.array_equal(np.asarray(out[f][:n_out]), sp[f].astype(np.float32)), f
    # unsplit rows are the input, bit for bit
    keep = ~flags_g
    for f in ("means", "log_scales", "opacity_logit"):
        assert np.array_equal(np.asarray(out[f][:n])[keep], getattr(scene, f)[keep]), f
    if not flags_g.any():
        return flags_g
    # a sign flip of v (allowed on a near-tie of its two largest components) swaps the pair
    flip = np.zeros(n, bool)
    if v_gpu is not None:
        dots = np.sum(np.asarray(v_gpu, np.float64) * v_o, axis=1)
        flip = flags_g & gap & (dots < 0)
        if flip.any():
            a = np.sort(np.abs(v_o[flip]), axis=1)
            assert np.all(a[:, -1] - a[:, -2] <= 1e-4), "eigenvector sign differs without a near-tie"
    split_idx = np.nonzero(flags_g)[0]
    app = n + np.arange(split_idx.size)                # row of each - offspring
    want = {k: np.array(sp[k], np.float64) for k in ("means", "log_scales", "opacity_logit")}
    fl = split_idx[flip[split_idx]]
    if fl.size:
        ap = app[flip[split_idx]]
        for k in want:
            want[k][fl], want[k][ap] = want[k][ap].copy(), want[k][fl].copy()
    s_max = float(np.exp(scene.log_scales.astype(np.float64)).max())
    tol = 1e-4 * step_scale * s_max + 1e-6
    om = np.asarray(out["means"][:n_out], np.float64)
    uniq = gap[split_idx]
    rows = np.concatenate([split_idx[uniq], app[uniq]])
    if rows.size:
        assert np.abs(om[rows] - want["means"][rows]).max() < tol
    # every pair, unique eigenvector or not: symmetric about its parent, offset eps_i |v|
    p = scene.means[split_idx].astype(np.float64)
    mid = 0.5 * (om[split_idx] + om[app])
    assert np.abs(mid - p).max() < 1e-6 + 1e-6 * np.abs(p).max()
    eps_i = step_scale * np.exp(scene.log_scales[split_idx].astype(np.float64)).max(axis=1)
    half = 0.5 * np.linalg.norm(om[split_idx] - om[app], axis=1)
    if dim == 3:
        assert np.all(np.abs(half - eps_i) <= 1e-4 * eps_i + 1e-6)
    else:
        assert np.all(half <= eps_i * (1 + 1e-4) + 1e-6)
    ol = np.asarray(out["opacity_logit"][:n_out], np.float64)
    both = np.concatenate([split_idx, app])
    if dim == 3:
        assert np.abs(ol[both] - want["opacity_logit"][both]).max() < 1e-5
    elif rows.size:
        o_g = 1 / (1 + np.exp(-ol[rows]))
        o_o = 1 / (1 + np.exp(-want["opacity_logit"][rows]))
        assert np.abs(o_g - o_o).max() < 1e-5
    if dim == 7:
        ls = np.asarray(out["log_scales"][:n_out], np.float64)
        if rows.size:
            assert np.abs(ls[rows] - want["log_scales"][rows]).max() < tol
        lp = scene.log_scales[split_idx].astype(np.float64)
        assert np.abs(0.5 * (ls[split_idx] + ls[app]) - lp).max() < 1e-6 + 1e-6 * np.abs(lp).max()
    return flags_g


def gpu_out(db, n_out):
    """The GPU split's output fields as numpy arrays."""
    return {f: getattr(db.out, f)[:n_out].cpu().numpy()
            for f in ("means", "log_scales", "quats", "opacity_logit", "sh")}
