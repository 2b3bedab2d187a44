"""Host logic of bench.py that needs no GPU: the clock record parsed from
nvidia-smi's CSV, the DRAM-traffic figure's source guard and the algorithmic
byte count."""
import hashlib
import os

import bench


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = lines
    return s


def _row(sm, mx=2070, active="0x0000000000000000", hw="Not Active", hwt="Not Active", swt="Not Active",
         cap="Not Active"):
    return f"0, {sm}, {mx}, 900.00, {active}, {hw}, {hwt}, {swt}, {cap}"


def test_clock_summary_median_under_load_and_reasons():
    lines = [_row(345), _row(1965), _row(1980), _row(1995, cap="Active"), _row(2010), "garbage", "0, [N/A], x"]
    c = _sampler(lines).summary()
    assert c["sm_max_mhz"] == 2070.0
    assert c["sm_mhz"] == 1987.5                  # idle samples (below 30 % of max) left out
    assert c["reasons"] == ["sw_power_cap"]
    assert c["samples"] == 5


def test_clock_summary_reports_every_throttle_reason():
    c = _sampler([_row(1500, hw="Active", hwt="Active", swt="Active")]).summary()
    assert c["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    c = _sampler([]).summary()
    assert c["sm_mhz"] is None and c["samples"] == 0 and c["reasons"] == []


def test_traffic_figure_only_for_the_profiled_sources():
    """The ncu DRAM traffic of the backward call is reported only while the
    sources of its three kernels and their launcher are the ones it was
    captured from (first 16 hex digits of their concatenated SHA-256)."""
    h = hashlib.sha256()
    for name in ("render.cu", "project.cu", "api.cu"):
        with open(os.path.join(bench.ROOT, "paper_2505_05587_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    got = bench._render_bwd_traffic()
    if h.hexdigest()[:16] == bench.RENDER_BWD_TRAFFIC["sources_sha256"]:
        assert got == bench.RENDER_BWD_TRAFFIC["bytes"]
    else:
        assert got is None
    assert os.path.exists(os.path.join(bench.ROOT, bench.RENDER_BWD_TRAFFIC["profile"]))


def test_algorithmic_bytes_per_unit():
    """The stage table's per-unit sums: 940 B per Gaussian, 124 per instance,
    76 per pixel, 8 per tile; the parameter record it assumes is the float32
    size of one SH-degree-3 Gaussian; the count is linear in each unit."""
    import synth
    sc = synth.cluster_scene(0, 4, 3)
    params = sum(a[0].nbytes for a in (sc.means, sc.log_scales, sc.quats, sc.opacity_logit, sc.sh))
    assert params == 236
    assert bench.ALGORITHMIC_BYTES[0][1] == params + 48          # parameters read, projected state written
    unit = [bench.algorithmic_bytes(*e) for e in ((1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1))]
    assert unit == [940, 124, 76, 8]
    assert bench.algorithmic_bytes(2, 3, 5, 7) == 2 * 940 + 3 * 124 + 5 * 76 + 7 * 8


def _reference_line(monkeypatch, per_full_s, steps=2, warmup=3):
    """The oracle arm's JSON line with the oracle replaced by a clock: a full
    iteration advances it by per_full_s, a strip of h rows by
    per_full_s * (0.05 + 0.95 h / HEIGHT)."""
    import contextlib
    import io
    import json
    t = [0.0]

    def fake_iteration(scene, cam, st, target, rows=None, all_cores=False):
        frac = 1.0 if rows is None else 0.05 + 0.95 * rows[1] / bench.HEIGHT
        t[0] += per_full_s * frac

    class Scene:
        n = 4

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setattr(bench, "_oracle_iteration", fake_iteration)
    monkeypatch.setattr(bench.time, "perf_counter", lambda: t[0])
    monkeypatch.setattr(bench.synth, "cluster_scene", lambda *a, **k: Scene())
    monkeypatch.setattr(bench.synth, "target_image", lambda *a, **k: None)

    class Args:
        pass

    Args.steps, Args.warmup = steps, warmup
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(Args())
    return json.loads(buf.getvalue().strip().splitlines()[-1])


def test_reference_arm_times_whole_iterations_when_they_fit(monkeypatch):
    out = _reference_line(monkeypatch, per_full_s=2.0)
    assert out["impl"] == "reference" and out["cpu_baseline"]["measured"] is True
    assert abs(out["value"] - 2000.0) < 1e-6
    assert out["e2e"]["value"] == out["value"] and out["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_extrapolates_strips_when_whole_iterations_do_not_fit(monkeypatch):
    out = _reference_line(monkeypatch, per_full_s=100.0, steps=5, warmup=3)
    assert out["cpu_baseline"]["measured"] is False
    assert "extrapolated" in out["cpu_baseline"]["sample"]
    # the fake's strip cost is linear in the rows, so the extrapolation is exact
    assert abs(out["value"] - 100_000.0) < 1e-3 * 100_000.0
