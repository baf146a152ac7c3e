"""bench.py's reference arm (the oracle timed on the host cores) on the CPU:
its one JSON line carries every key of the bench contract, and ranks other
than 0 under a launcher print nothing and exit 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, *args):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)


def test_reference_arm_line_has_the_contract_keys():
    r = _run({}, "--workload", "c1", "--steps", "2", "--warmup", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "events/s" and d["steps"] == 2 and d["warmup"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_print_nothing():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"}, "--workload", "c1", "--steps", "1", "--warmup", "0")
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_roofline_counts_the_algorithmic_bytes_of_the_measurement_rule():
    # 16 B per event and one complex64 coefficient write per mode and asset
    # are algorithmic; records and grid rows are implementation bytes
    sys.path.insert(0, ROOT)
    import bench
    stage_ms = {"prep": 0.013, "spread": 0.024, "fft": 0.031, "gram": 0.016, "reduce": 0.007, "setup": 0.5,
                "fft_cols": 0.0, "fft_rows": 0.0, "fused": 0.0}
    n, D, N, Mr = 766162, 100, 10000, 40500
    roof = bench.hbm_roofline(stage_ms, n, D, N, Mr, False, {"hbm_gbs": 6792.7}, "measured", ("c3", "bf16x3", "es"))
    assert roof["kernel"] == "fft"
    assert roof["algorithmic_bytes_per_launch"] == 8.0 * (N + 1) * D
    assert roof["implementation_bytes_per_launch"] == 4.0 * Mr * D
    assert abs(roof["achieved"] - 8.0 * (N + 1) * D / 0.031e-3 / 1e9) < 1e-6
    assert abs(roof["frac"] - roof["achieved"] / 6792.7) < 1e-12
    ch = roof["chain"]
    assert ch["kernels"] == ["prep", "spread", "fft"]
    assert abs(ch["ms"] - 0.068) < 1e-12
    assert ch["algorithmic_bytes"] == 16.0 * n + 8.0 * (N + 1) * D
    assert ch["implementation_bytes"] == 12.0 * n + (12.0 * n + 4.0 * Mr * D) + 4.0 * Mr * D
    # the spreading kernel moves no algorithmic bytes of its own
    slow = dict(stage_ms, spread=0.05)
    assert bench.hbm_roofline(slow, n, D, N, Mr, False, {"hbm_gbs": 6792.7}, "m", ("c3", "bf16x3", "es"))["frac"] == 0.0
    # FP64: complex128 coefficients
    r64 = bench.hbm_roofline(stage_ms, n, D, N, Mr, True, {"hbm_gbs": 6792.7}, "m", ("c3", "fp64", "es"))
    assert r64["algorithmic_bytes_per_launch"] == 16.0 * (N + 1) * D
