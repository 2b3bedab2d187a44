"""Writes the oracle-derived golden fixture of the tiny scene.

Every stored value comes from the float64 CPU oracle (``oracle/``) on inputs
drawn by ``synth``; nothing here runs the CUDA path.  The fixture lets the CPU
suite notice any change of the oracle's arithmetic (the stored values stop
matching) and lets a GPU test compare the CUDA path with fixed numbers.

Workload: the tiny scene (256 Gaussians, SH degree 0, seed 0), one 64x64 view
with fx = 64 looking down +z, 16x16 tiles and the default rasterisation
constants, the uniform target of seed 2, one L1 iteration (Section 3, Eq. for
the loss), the backward with splitting matrices (Section 4.4, Algorithm 1), the
minimum eigenpairs by the trigonometric formula (Appendix on the
eigendecomposition) and the split at eps_split = 0 with step scale 1
(Theorem 2).

Run ``python tests/golden/make_golden.py`` from the repository root to rewrite
``tiny_64x64_seed0.json``.
"""
from __future__ import annotations

import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

FIXTURE = os.path.join(HERE, "tiny_64x64_seed0.json")
PIXEL_STRIDE = 8          # image samples on an 8 x 8 pixel lattice
ROW_STRIDE = 8            # per-Gaussian samples: every 8th Gaussian that any pixel reaches
EPS_SPLIT = 0.0
STEP_SCALE = 1.0


def tiny_case():
    scene = synth.tiny_scene(0)
    cam = synth.camera_identity(64, 64, 64.0)
    st = synth.Settings()
    target = synth.target_image(2, cam.height, cam.width)
    return scene, cam, st, target


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def pack_bits(mask: np.ndarray) -> str:
    return np.packbits(np.asarray(mask, bool).reshape(-1)).tobytes().hex()


def unpack_bits(hexstr: str, count: int) -> np.ndarray:
    return np.unpackbits(np.frombuffer(bytes.fromhex(hexstr), np.uint8))[:count].astype(bool)


def upper6(S: np.ndarray) -> np.ndarray:
    return np.stack([S[:, 0, 0], S[:, 0, 1], S[:, 0, 2], S[:, 1, 1], S[:, 1, 2], S[:, 2, 2]], 1)


def compute() -> dict:
    """The fixture's contents, computed by the oracle."""
    scene, cam, st, target = tiny_case()
    isg = oracle.integer_stage(scene, cam, st)
    keys, gids, ranges = oracle.bin_sort(scene, cam, st)
    ref = oracle.render(scene, cam, st)
    loss, dL = oracle.l1_loss_grad(ref["image"], target)
    if np.any(dL == 0.0):
        raise RuntimeError("a channel equals its target; the L1 sign is undefined there")
    # both sides of the comparison take dL/dC rounded to float32
    dL32 = dL.astype(np.float32).astype(np.float64)
    acc = oracle.backward(scene, cam, st, dL32)
    lam, v = oracle.eig3_min(acc["S"], 1.0)
    sp = oracle.split(scene, lam, v, EPS_SPLIT, STEP_SCALE)

    ys = np.arange(0, cam.height, PIXEL_STRIDE)
    xs = np.arange(0, cam.width, PIXEL_STRIDE)
    pixels = [[int(y), int(x), *[float(c) for c in ref["image"][y, x]], float(ref["final_T"][y, x]),
               int(ref["n_contrib"][y, x]), bool(ref["band"][y, x])] for y in ys for x in xs]
    reached = np.nonzero(isg["tiles"] > 0)[0]
    rows = []
    for i in reached[::ROW_STRIDE]:
        rows.append({"i": int(i),
                     "S": [float(x) for x in upper6(acc["S"][i:i + 1])[0]],
                     "S_po": [float(x) for x in acc["S_po"][i]],
                     "grad_means": [float(x) for x in acc["means"][i]],
                     "grad_log_scales": [float(x) for x in acc["log_scales"][i]],
                     "grad_quats": [float(x) for x in acc["quats"][i]],
                     "grad_opacity_logit": float(acc["opacity_logit"][i]),
                     "grad_sh": [float(x) for x in acc["sh"][i].reshape(-1)],
                     "lambda_min": float(lam[i]),
                     "v_min": [float(x) for x in v[i]]})
    return {
        "workload": {"scene": "synth.tiny_scene(0)  (256 Gaussians, SH degree 0)",
                     "camera": "synth.camera_identity(64, 64, 64.0)",
                     "settings": "synth.Settings()  (16x16 tiles)",
                     "target": "synth.target_image(2, 64, 64)",
                     "eps_split": EPS_SPLIT, "step_scale": STEP_SCALE, "T_split": 1},
        "integer": {"instances": int(len(keys)),
                    "tiles_touched": [int(t) for t in isg["tiles"]],
                    "keys_sha256": sha256(keys.astype(np.uint64)),
                    "gids_sha256": sha256(gids.astype(np.uint32)),
                    "ranges_sha256": sha256(ranges.astype(np.uint32))},
        "pixel_stride": PIXEL_STRIDE,
        "pixels": pixels,
        "loss": float(loss),
        "dL_positive_bits": pack_bits(dL > 0),
        "dL_magnitude": float(np.abs(dL).max()),
        "row_stride": ROW_STRIDE,
        "rows": rows,
        "lambda_min": [float(x) for x in lam],
        "split": {"flags_bits": pack_bits(sp["flags"]), "n_out": int(sp["n_out"]),
                  "parent": [int(p) for p in sp["parent"][scene.n:]]},
    }


def dump(data: dict) -> str:
    """JSON with one top-level key per line and one list item per line."""
    out = []
    for k, val in data.items():
        if isinstance(val, list) and val and isinstance(val[0], (list, dict)):
            items = ",\n".join(json.dumps(x, separators=(",", ":")) for x in val)
            out.append(f"{json.dumps(k)}:[\n{items}]")
        else:
            out.append(f"{json.dumps(k)}:{json.dumps(val, separators=(',', ':'))}")
    return "{\n" + ",\n".join(out) + "\n}\n"


def main():
    data = compute()
    with open(FIXTURE, "w") as f:
        f.write(dump(data))
    print(f"wrote {FIXTURE}: {os.path.getsize(FIXTURE)} bytes, {len(data['rows'])} sampled Gaussians, "
          f"{data['split']['n_out'] - 256} splits")


if __name__ == "__main__":
    main()
