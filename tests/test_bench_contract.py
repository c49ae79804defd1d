"""The benchmark's JSON contract on the host (no GPU): the reference arm's line
(the FP64 oracle timed on the host cores), the silent exit of non-zero ranks,
the DRAM-traffic figure tied to the kernel source it was captured on, and the
roofline peak's provenance."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _run_bench(*args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_line_has_the_contract_keys():
    p = _run_bench("--impl", "reference", "--steps", "2", "--warmup", "1")
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["higher_is_better"] is False
    assert d["warmup"] >= 3                      # at least 3 warm-up steps, whatever was asked
    assert d["value"] > 0 and d["unit"] == "us"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    p = _run_bench("--impl", "reference", "--steps", "2", "--warmup", "1",
                   env_extra={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert not [l for l in p.stdout.splitlines() if l.startswith("{")]


def test_traffic_is_reported_only_for_the_captured_kernel_source(monkeypatch):
    import bench
    rec = dict(bench.NCU_TRAFFIC)
    got = bench.fused_traffic()
    assert got in (None, rec["dram_bytes"])
    monkeypatch.setitem(bench.NCU_TRAFFIC, "fused_cu_sha256", "0" * 16)
    assert bench.fused_traffic() is None            # another kernel source: no traffic claimed
    sha = bench.fused_source_sha()
    monkeypatch.setitem(bench.NCU_TRAFFIC, "fused_cu_sha256", sha[:16])
    assert bench.fused_traffic() == rec["dram_bytes"]
    # the committed summary the figure comes from exists and names the same source
    with open(os.path.join(ROOT, rec["summary"])) as f:
        assert rec["fused_cu_sha256"] in f.read()


def test_peak_provenance(monkeypatch, tmp_path):
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peak, kind = bench.measured_peaks()
    assert peak == 6400.0 and kind.startswith("of fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7100.0}))
    peak, kind = bench.measured_peaks()
    assert peak == 7100.0 and kind.startswith("of measured")


def test_roofline_block_is_against_the_measured_l2():
    import bench
    from paper_2009_00946_b300 import configs
    cfg = configs.c2_elt()
    l2 = {"read_gbs": 20000.0, "copy_gbs": 16000.0, "bytes": 48 << 20, "passes": 40, "reps": 5}
    r = bench.roofline_block(cfg, 100.0, 20.0, l2, 6500.0, "of measured", None)
    assert r["bound"] == "l2" and r["unit"] == "GB/s" and r["peak"] == 20000.0   # the larger L2 figure
    alg = bench.algorithmic_bytes_per_frame(cfg, bench.N_ITER)
    assert abs(r["achieved"] - alg / 100e-6 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 20000.0) < 1e-12
    # one PCG iteration: 16 N + 4 NW FP32 elements (N = 9 * 128^2, NW = 6 * 85^2)
    it = r["per_iteration"]
    assert it["algorithmic_bytes"] == 4 * (16 * 9 * 128 ** 2 + 4 * 6 * 85 ** 2)
    assert abs(it["frac"] - it["algorithmic_bytes"] / 20e-6 / 1e9 / 20000.0) < 1e-12
    assert abs(r["hbm"]["frac"] - r["achieved"] / 6500.0) < 1e-12
    assert r["peak_kind"].startswith("of measured")


if __name__ == "__main__":
    sys.exit(pytest.main([__file__, "-q"]))
