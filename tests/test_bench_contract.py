"""The reference arm of bench.py (the FP64 oracle on the host cores) prints the one JSON line of the
benchmark contract; checked on a tiny sample on CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--worlds", "16", "--ref-sample", "4", "--iters", "200"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] >= 1


def test_recorded_step_kernel_traffic_belongs_to_the_sources():
    """The DRAM traffic that the bench line reports comes from an ncu capture recorded with the
    SHA-256 of the step kernel's sources: it is used, scaled by worlds, only while it belongs to the
    sources in the tree; after a kernel edit without a new capture the bench reports it as null."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    entry = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["biped"]
    got = bench.step_kernel_traffic("biped", 4096)
    if entry["source_sha256"] == bench.kernel_source_hash():
        assert got == entry["dram_bytes"] * 4096 / entry["worlds"]
        assert got / 4096 < 16384       # bytes per world-step: everything else stays on chip
    else:
        assert got is None


def test_hbm_roofline_of_the_step_kernel():
    """The bench line's HBM entry: DRAM bytes per launch over the launch time against the measured
    copy bandwidth; absent when either is unknown."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    h = bench.hbm_roofline(30.9e6, 21.06, {"hbm_gbs": 6701.2})
    assert abs(h["achieved"] - 30.9e6 / 0.02106 / 1e9) < 1e-9 and h["unit"] == "GB/s"
    assert abs(h["frac"] - h["achieved"] / 6701.2) < 1e-15 and h["frac"] < 1e-3     # far from the HBM bound
    assert bench.hbm_roofline(None, 21.06, {"hbm_gbs": 6701.2}) is None
    assert bench.hbm_roofline(30.9e6, 21.06, {}) is None
