"""The oracle against its stored golden fixture (tests/golden/).

The fixture was written by tests/golden/make_golden.py, which calls only the
oracle.  Recomputing it must give the stored integers, hashes and decisions
exactly and the stored floats to float64 rounding, so that any change of the
oracle's arithmetic shows here and has to come with a regenerated fixture.
The fixture's decisions are also checked against the rules they follow
(Theorem 2's split condition, the compaction order of Algorithm 1)."""
import importlib.util
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def _make_golden():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def stored():
    with open(os.path.join(GOLDEN, "tiny_64x64_seed0.json")) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def mg():
    return _make_golden()


def _close(a, b, rtol=1e-12):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = max(float(np.abs(b).max()), 1e-300) if b.size else 1.0
    return a.shape == b.shape and bool(np.all(np.abs(a - b) <= rtol * (np.abs(b) + scale)))


def test_oracle_reproduces_the_fixture(stored, mg):
    got = mg.compute()
    assert got["workload"] == stored["workload"]
    assert got["integer"] == stored["integer"]
    assert got["dL_positive_bits"] == stored["dL_positive_bits"]
    assert got["split"] == stored["split"]
    assert _close(got["loss"], stored["loss"])
    assert _close(got["dL_magnitude"], stored["dL_magnitude"])
    gp, sp = np.array(got["pixels"], np.float64), np.array(stored["pixels"], np.float64)
    assert np.array_equal(gp[:, [0, 1, 6, 7]], sp[:, [0, 1, 6, 7]])     # positions, counts, band flags
    assert _close(gp[:, 2:6], sp[:, 2:6])
    assert _close(got["lambda_min"], stored["lambda_min"])
    assert [r["i"] for r in got["rows"]] == [r["i"] for r in stored["rows"]]
    for key in ("S", "S_po", "grad_means", "grad_log_scales", "grad_quats", "grad_opacity_logit", "grad_sh",
                "lambda_min", "v_min"):
        assert _close([r[key] for r in got["rows"]], [r[key] for r in stored["rows"]]), key


def test_fixture_decisions_follow_the_split_rule(stored, mg):
    """Flags are lambda_min < eps_split (Theorem 2); the appended offspring's
    parents are the flagged indices in increasing order; N' = N + #flags."""
    lam = np.array(stored["lambda_min"])
    n = lam.size
    flags = mg.unpack_bits(stored["split"]["flags_bits"], n)
    assert np.array_equal(flags, lam < stored["workload"]["eps_split"])
    assert stored["split"]["parent"] == [int(i) for i in np.nonzero(flags)[0]]
    assert stored["split"]["n_out"] == n + int(flags.sum())


def test_fixture_integer_stage_is_consistent(stored):
    """The instance count is the sum of the tiles each Gaussian touches."""
    assert stored["integer"]["instances"] == sum(stored["integer"]["tiles_touched"])


def test_fixture_pixels_are_consistent(stored):
    """Colours are non-negative, transmittance lies in (0, 1], and a pixel
    that no Gaussian reaches keeps the black background with T = 1."""
    px = np.array(stored["pixels"], np.float64)
    assert np.all(px[:, 2:5] >= 0.0)
    assert np.all((px[:, 5] > 0.0) & (px[:, 5] <= 1.0))
    empty = px[:, 6] == 0
    assert np.all(px[empty, 2:5] == 0.0) and np.all(px[empty, 5] == 1.0)


def test_fixture_eigenpairs_are_eigenpairs(stored):
    """For every sampled Gaussian: S v = lambda_min v, |v| = 1, and lambda_min
    is the smallest eigenvalue of S (LAPACK's symmetric solver)."""
    for r in stored["rows"]:
        a, b, c, d, e, f = r["S"]
        S = np.array([[a, b, c], [b, d, e], [c, e, f]])
        v = np.array(r["v_min"])
        nrm = max(np.linalg.norm(S), 1e-300)
        assert abs(np.linalg.norm(v) - 1.0) < 1e-12
        assert np.linalg.norm(S @ v - r["lambda_min"] * v) <= 1e-10 * nrm
        assert abs(np.linalg.eigvalsh(S)[0] - r["lambda_min"]) <= 1e-10 * nrm
