"""bench.py on the CPU: the reference arm's JSON line and the algorithmic-byte model.

The reference arm times the FP64 oracle on the host.  Here it runs on a tiny
sample, checked key by key against the benchmark contract.  The model
behind the roofline's ``achieved`` figure is checked term by term against the
per-unit byte counts it documents.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(args, **env):
    e = dict(os.environ, PG_ORACLE_SAMPLE_NX="24", PG_ORACLE_SAMPLE_STEPS="4", **env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True,
                          text=True, timeout=300, env=e, cwd=ROOT)


def test_reference_arm_line():
    r = _run(["--impl", "reference", "--steps", "2", "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "steps/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 1)
    assert d["ms_per_step"] > 0 and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_are_silent():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"], RANK="1", WORLD_SIZE="2")
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_algorithmic_byte_model():
    n, mn, n_src = 1000, 2.5, 30
    ab = bench.algorithmic_bytes
    base = ab({"total_sweeps": 0, "total_outer": 0}, n, mn, n_src, True, 0)
    assert base == 0.0
    # one FP32 sweep: 16 + 4 m/n per node (point form), 20 + 4 m/n (column blocks)
    assert ab({"total_sweeps": 1, "total_outer": 0}, n, mn, n_src, True, 0) == (16 + 4 * mn) * n
    assert ab({"total_sweeps": 1, "total_outer": 0, "lattice_sweeps": 3}, n, mn, n_src, True, 0) == (20 + 4 * mn) * n
    # one FP64 sweep: 32 + 8 m/n
    assert ab({"total_sweeps": 1, "total_outer": 0}, n, mn, n_src, False, 0) == (32 + 8 * mn) * n
    # one outer pass: 52 (mixed) or 56 (FP64) + 8 m/n, plus 16 for the carried M d
    assert ab({"total_sweeps": 0, "total_outer": 1}, n, mn, n_src, True, 0) == (52 + 8 * mn + 16) * n
    assert ab({"total_sweeps": 0, "total_outer": 1}, n, mn, n_src, False, 0) == (56 + 8 * mn + 16) * n
    # steps: one full start in 16 (56 + 8 + 8 m/n), the rest incremental (72), plus the
    # step end (8 per node) and 56 B per PWL source
    one = ab({"total_sweeps": 0, "total_outer": 0}, n, mn, n_src, True, 1)
    assert one == pytest.approx((56 + 8 + 8 * mn) * n + 56 * n_src + 8 * n)
    sixteen = ab({"total_sweeps": 0, "total_outer": 0}, n, mn, n_src, True, 16)
    assert sixteen == pytest.approx((56 + 8 + 8 * mn) * n + 15 * 72 * n + 16 * (56 * n_src + 8 * n))


def test_survey_byte_model():
    """The roofline's byte model, term by term: 16 + 4 m/n per FP32 node-sweep (32 + 8 m/n
    in FP64), 24 + 8 m/n per node per FP64 residual pass, 24 B per node plus 36 B per
    source per step.  The column-block form counts as an FP32 sweep."""
    n, mn, n_src = 1000, 2.5, 30
    sb = bench.survey_bytes
    z = {"total_sweeps": 0, "total_outer": 0}
    assert sb(z, n, mn, n_src, True, 0) == 0.0
    assert sb({"total_sweeps": 1, "total_outer": 0}, n, mn, n_src, True, 0) == (16 + 4 * mn) * n
    assert sb({"total_sweeps": 1, "total_outer": 0, "lattice_sweeps": 3}, n, mn, n_src, True, 0) == (16 + 4 * mn) * n
    assert sb({"total_sweeps": 1, "total_outer": 0}, n, mn, n_src, False, 0) == (32 + 8 * mn) * n
    assert sb({"total_sweeps": 0, "total_outer": 1}, n, mn, n_src, True, 0) == (24 + 8 * mn) * n
    assert sb(z, n, mn, n_src, True, 7) == 7 * (24 * n + 36 * n_src)


def test_config3_sample_choice():
    """The per-config bench compares three grids of the batch with the oracle: the smallest
    single-layer grid, the smallest two-layer grid and the single-layer grid nearest 256."""
    import pgsynth
    shapes = pgsynth.config3_shapes()
    pick = bench._c3_sample(shapes)
    assert len(pick) == 3
    one = [s for s, l in shapes if l == 1]
    assert min(one) in [shapes[k][0] for k in pick if shapes[k][1] == 1]
    assert any(shapes[k][1] == 2 and shapes[k][0] == min(s for s, l in shapes if l == 2) for k in pick)
