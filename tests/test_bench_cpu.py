"""Host-side pieces of bench.py, on the CPU: the committed ncu traffic figures
are used only while the profiled kernel sources are unchanged, and the
reference arm (the oracle on the host cores) prints one JSON line with the
keys the measurement contract asks for."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_traffic_figures_only_for_unchanged_sources(tmp_path):
    b = load_bench()
    sources = ["dvbm_device.cuh", "dvbm_step.cu"]
    entry = {"source_hash": b.kernel_source_hash(tuple(sources)), "sources": sources, "dram_bytes_per_cell": 1.0}
    for e, used in ((entry, True), (dict(entry, source_hash="0" * 16), False)):
        p = tmp_path / "traffic.json"
        p.write_text(json.dumps({"k_step_fp64": e}))
        b.PROFILE_TRAFFIC = str(p)
        assert (b.profile_traffic("k_step_fp64") is not None) == used
    assert b.profile_traffic("no_such_kernel") is None


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--cpu-sample", "32", "--steps", "2",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == "MLUPS" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 2 and line["warmup"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and "32x32" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
