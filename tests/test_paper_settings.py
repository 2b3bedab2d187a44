"""The constants the paper fixes (tests/golden/paper_hyperparameters.json, each
with its source) against the trainer's defaults and schedule, and against the
oracle's split rule."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def paper():
    with open(os.path.join(HERE, "golden", "paper_hyperparameters.json")) as f:
        return json.load(f)


def test_trainer_defaults_are_the_papers(paper):
    pytest.importorskip("torch")
    from paper_2505_05587_gb300.train import TrainConfig
    cfg = TrainConfig()
    assert cfg.start == paper["densify_start_step"]
    assert cfg.T_split == paper["densify_every_steps"]
    assert cfg.eps_split == paper["eps_split"]


def test_densification_schedule(paper):
    pytest.importorskip("torch")
    from paper_2505_05587_gb300.train import TrainConfig, densify_due
    cfg = TrainConfig()
    due = [t for t in range(1, 2001) if densify_due(t, cfg)]
    start, every = paper["densify_start_step"], paper["densify_every_steps"]
    assert due == list(range(start, 2001, every))
    assert due[0] == 500 and len(due) == 16


def test_oracle_split_makes_two_half_opacity_offspring(paper):
    """Gaussians with lambda_min < eps_split become exactly two rows at
    p +- eps v_min, each with opacity o * 1/2; the others are copied."""
    sc = synth.tiny_scene(4, 40)
    rng = np.random.default_rng(4)
    lam = rng.uniform(-1.0, 1.0, sc.n)
    lam[::7] = paper["eps_split"]                   # on the threshold: strict inequality keeps them
    v = rng.standard_normal((sc.n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    out = oracle.split(sc, lam, v, paper["eps_split"], step_scale=0.5)
    flagged = np.nonzero(lam < paper["eps_split"])[0]
    assert out["n_out"] == sc.n + len(flagged)
    rows_per_parent = np.bincount(out["parent"], minlength=sc.n)
    assert np.all(rows_per_parent[flagged] == paper["offspring_per_split"])
    assert np.all(np.delete(rows_per_parent, flagged) == 1)
    o = 1.0 / (1.0 + np.exp(-sc.opacity_logit.astype(np.float64)))
    o_out = 1.0 / (1.0 + np.exp(-out["opacity_logit"]))
    eps = 0.5 * np.exp(sc.log_scales.astype(np.float64)).max(axis=1)
    for r, i in enumerate(flagged):
        j = sc.n + r
        for row, sgn in ((i, 1.0), (j, -1.0)):
            assert abs(o_out[row] - paper["offspring_opacity_factor"] * o[i]) <= 1e-6 * o[i]
            assert np.allclose(out["means"][row], sc.means[i] + sgn * eps[i] * v[i], rtol=0, atol=1e-6)
        # the pair's weighted mean displacement vanishes (w = 1/2 each)
        w = paper["offspring_weight"]
        assert np.allclose(w * out["means"][i] + w * out["means"][j], sc.means[i], rtol=0, atol=1e-6)
