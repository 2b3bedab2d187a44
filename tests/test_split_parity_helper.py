"""The split parity check itself, on the CPU: a split written from the
oracle's own output (rounded to float32 as the GPU stores it) passes, and
planted mistakes in the compaction or the offspring fail it."""
import numpy as np
import pytest

import oracle
import synth

import split_parity as SP


def _case():
    sc = synth.tiny_scene(0)
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings()
    r = oracle.render(sc, cam, st)
    _, g = oracle.l1_loss_grad(r["image"], synth.target_image(2, 64, 64))
    S = oracle.backward(sc, cam, st, g)["S"]
    lam, v = oracle.eig3_min(S)
    nrm = np.linalg.norm(S.reshape(-1, 9), axis=1)
    ev = np.linalg.eigvalsh(S)
    gap = (ev[:, 1] - ev[:, 0]) > 1e-3 * nrm
    decided = np.abs(lam) > 1e-6 * np.maximum(nrm, 1e-30)
    sp = oracle.split(sc, lam, v, 0.0, 0.5)
    out = {f: sp[f].astype(np.float32) for f in ("means", "log_scales", "quats", "opacity_logit", "sh")}
    return sc, lam, v, gap, decided, sp, out


def test_oracle_split_as_float32_passes():
    sc, lam, v, gap, decided, sp, out = _case()
    assert sp["flags"].sum() > 0
    f = SP.check_split(sc, out, sp["parent"], sp["n_out"], lam, v, sp["flags"], decided, gap, 0.0, 0.5, v_gpu=v)
    assert np.array_equal(f, sp["flags"])


def test_planted_mistakes_fail():
    sc, lam, v, gap, decided, sp, out = _case()
    n, n_out = sc.n, sp["n_out"]
    # two appended rows swapped (their parents and their rows together)
    par = sp["parent"].copy()
    o2 = {k: a.copy() for k, a in out.items()}
    a, b = n, n + 1
    par[[a, b]] = par[[b, a]]
    for k in o2:
        o2[k][[a, b]] = o2[k][[b, a]]
    with pytest.raises(AssertionError):
        SP.check_split(sc, o2, par, n_out, lam, v, sp["flags"], decided, gap, 0.0, 0.5, v_gpu=v)
    # an offspring displaced with the wrong sign
    i = int(np.flatnonzero(sp["flags"] & gap)[0])
    o3 = {k: a.copy() for k, a in out.items()}
    o3["means"][i] = (2 * sc.means[i].astype(np.float64) - sp["means"][i]).astype(np.float32)
    with pytest.raises(AssertionError):
        SP.check_split(sc, o3, sp["parent"], n_out, lam, v, sp["flags"], decided, gap, 0.0, 0.5, v_gpu=v)
    # a decided Gaussian left unsplit
    j = int(np.flatnonzero(sp["flags"] & decided)[0])
    f4 = sp["flags"].copy()
    f4[j] = False
    s4 = oracle.split(sc, lam, v, 0.0, 0.5, flags=f4)
    o4 = {f: s4[f].astype(np.float32) for f in out}
    with pytest.raises(AssertionError):
        SP.check_split(sc, o4, s4["parent"], s4["n_out"], lam, v, sp["flags"], decided, gap, 0.0, 0.5, v_gpu=v)
    # a copied attribute altered
    o5 = {k: a.copy() for k, a in out.items()}
    o5["sh"][n_out - 1] += 1.0
    with pytest.raises(AssertionError):
        SP.check_split(sc, o5, sp["parent"], n_out, lam, v, sp["flags"], decided, gap, 0.0, 0.5, v_gpu=v)
