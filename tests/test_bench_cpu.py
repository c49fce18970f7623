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


def _free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = load_bench()
        t = b.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")  # rank 1 is the slow one
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
            json.dump({"t": t, "mlups": b.whole_job_mlups(4096 * 4096, 20, world, t)}, fh)
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_every_grid(tmp_path):
    """Replicas on two gloo ranks: each rank's timed region is reduced to the
    slowest rank's, and the throughput counts the cells of both grids."""
    import torch.multiprocessing as mp
    mp.start_processes(_rank_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert got[0] == got[1]
    assert got[0]["t"] == 15.0
    assert abs(got[0]["mlups"] - 4096 * 4096 * 20 * 2 / 15.0 / 1e6) < 1e-9


def test_reference_arm_under_torchrun_prints_once():
    """Launched as the driver launches N > 1 (torch.distributed.run, two ranks),
    the reference arm runs on rank 0 alone: one JSON line, both ranks exit 0."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--cpu-sample", "32", "--steps", "1", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
