#!/usr/bin/env python3
"""Benchmark of the GB300 DVBM time step (one JSON line on rank 0).

Workload: periodic 4096 x 4096 random-phase multimode flow (Gaussian shell
spectrum peaking at |k| = 8, rms Ma 0.3, rms dT 0.05, seed 0), Pr = 0.71,
gamma = 1.4, mu = 5e-5, D2Q25 split II.  A step is one full time step of the
hot path (moments, collision, advection, update, ghost layers).  ``value`` is
whole-job MLUPS of FP64 storage with the state resident in HBM; FP32-deviation
storage is measured on the same workload in ``fp32dev``.  The state (2 x 6.7 GB)
is far larger than L2, so no L2 flush is needed between steps.

``--impl reference`` times the FP64 CPU oracle (the reference arm) on host cores.
Under torchrun each rank runs an independent replica (weak scaling, no
collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_CELL = {"fp64": 2 * 50 * 8, "fp32dev": 2 * 50 * 4, "d2q16": 2 * 32 * 8}  # read + write all populations
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
FALLBACK_HBM_GBS = 6800.0
# GB300 unit counts and clock (profiling recipe): 152 SMs, 2.07 GHz; FP64 at 2
# instructions per clock per SM (FMA = 2 flops); 4 warp schedulers per SM,
# one warp instruction per scheduler per clock
NOMINAL_HBM_GBS = 8000.0  # the 8 TB/s nominal HBM3e figure the throughput target is stated against
NOMINAL_FP64_TFLOPS = 152 * 2 * 2.07e9 * 2 / 1e12          # 1.259
NOMINAL_ISSUE_GWARPINST = 152 * 4 * 2.07e9 / 1e9            # 1258.6 G warp instructions / s


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32dev", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=512, help="oracle sample grid size")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-d2q16", action="store_true")
    ap.add_argument("--no-workloads", action="store_true")
    ap.add_argument("--layout", default="slabs", choices=["slabs", "replicas"],
                    help="with several GPUs: one band of a y-decomposed grid per GPU, halo rows over NCCL (slabs), "
                         "or one independent grid per GPU (replicas)")
    ap.add_argument("--cpu-table", action="store_true",
                    help="the oracle's CPU baseline table on one and on all host threads (one JSON line)")
    ap.add_argument("--sweep", action="store_true",
                    help="throughput sweep over grid size, rms Mach number and storage form (one JSON line)")
    return ap.parse_args()


def workload_config(N, world=1, layout="slabs"):
    if world > 1 and layout == "slabs":
        par = (f"slabs along y: one {N}-row band per GPU of a periodic {N}x{N * world} grid (the {N}x{N} flow "
               f"repeated in y), two halo rows per side per step over NCCL send/recv, dt and totals all-reduced")
    else:
        par = "replicas (one independent grid per GPU)"
    return {"workload": f"periodic multimode flow {N}x{N}, rms Ma 0.3, seed 0 (throughput sweep)",
            "grid": [N, N], "lattice": "D2Q25", "energy_split": "II", "Pr": 0.71, "gamma": 1.4, "mu": 5e-5,
            "cfl": 0.01, "beta": 1.2, "l2": "state 2x50 planes x N^2 (> 129 MB L2): no flush needed",
            "parallelism": par}


STEP_KERNEL_SOURCES = ("dvbm_device.cuh", "dvbm_step.cu")


def kernel_source_hash(sources=STEP_KERNEL_SOURCES):
    """Hash of the sources a step kernel is compiled from (the committed ncu
    figures are only used while this hash matches)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2510_04197_gb300", "csrc")
    for fn in sources:
        h.update(open(os.path.join(d, fn), "rb").read())
    return h.hexdigest()[:16]


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (a job takes as long as its slowest rank);
    x itself without a process group."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def conservation_drift(t0, t1, steps):
    """Change of the domain totals (mass, x/y momentum, energy) over a run:
    mass and energy relative to their initial values, momentum per unit
    initial mass (a velocity, in units of sqrt(R T_ref))."""
    m0 = t0[0]
    return {"steps": steps, "mass": (t1[0] - t0[0]) / m0, "momentum_x": (t1[1] - t0[1]) / m0,
            "momentum_y": (t1[2] - t0[2]) / m0, "energy": (t1[3] - t0[3]) / t0[3]}


def whole_job_mlups(cells_per_rank, steps, world, seconds):
    """Cell updates of all ranks (one independent grid each) per second, in
    millions."""
    return cells_per_rank * steps * world / seconds / 1e6


def load_peaks():
    try:
        with open(PEAKS_FILE) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def profile_traffic(kernel_key):
    """DRAM bytes per cell of a kernel from the committed ncu summary, if it
    was taken on the current kernel sources; else None."""
    try:
        with open(PROFILE_TRAFFIC) as fh:
            t = json.load(fh)
        e = t.get(kernel_key)
        if e and e.get("source_hash") == kernel_source_hash(tuple(e.get("sources", STEP_KERNEL_SOURCES))):
            return e
    except Exception:
        pass
    return None


class ClockSampler:
    """Samples nvidia-smi clocks/throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_mlups(N, steps, warmup=1, threads=None, fields=None, P_kw=None, cfl=0.01):
    """MLUPS of the FP64 CPU oracle, as it stands, on an N^2 periodic field
    (default: the bench's multimode recipe), ``warmup`` untimed steps then
    ``steps`` timed; ``threads`` = torch intra-op threads (None: all)."""
    import torch
    from oracle import dvbm_oracle as O
    from paper_2510_04197_gb300 import inputs
    F = fields if fields is not None else inputs.multimode(N, seed=0, rms_Ma=0.3)
    t = lambda a: torch.tensor(a, dtype=torch.float64)
    P = O.Params(**(P_kw or dict(Pr=0.71, gamma=1.4, mu=5e-5)))
    old = torch.get_num_threads()
    if threads:
        torch.set_num_threads(threads)
    try:
        Ny, Nx = F.rho.shape
        sim = O.Simulation(O.Grid(Nx, Ny, F.Lx, F.Ly), P, t(F.rho), t(F.ux), t(F.uy), t(F.T), cfl=cfl)
        sim.run(warmup)
        t0 = time.perf_counter()
        sim.run(steps)
        el = time.perf_counter() - t0
        used = torch.get_num_threads()
    finally:
        torch.set_num_threads(old)
    return Nx * Ny * steps / el / 1e6, el, used


def cpu_baseline(N_sample, steps=30, warmup=1):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload:
    a periodic N_sample^2 multimode field of the same recipe, ``warmup``
    untimed steps, then ``steps`` timed steps on all host threads (512^2 x 30
    steps: about 12 s on 16 host cores); beside it one thread on a 256^2 x 4
    step sample."""
    v, el, used = oracle_mlups(N_sample, steps, warmup)
    v1, el1, _ = oracle_mlups(256, 4, 1, threads=1)
    return {"value": v, "unit": "MLUPS", "cores": used, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"{N_sample}x{N_sample} periodic multimode (same recipe), {steps} FP64 steps after {warmup} warm-up, "
                      f"{el:.1f} s on {used} threads",
            "single_thread": {"value": v1, "unit": "MLUPS", "cores": 1,
                              "sample": f"256x256, 4 FP64 steps after 1 warm-up, {el1:.1f} s"}}


def cpu_table():
    """The oracle's baseline table (one JSON line): config 1 (64^2 wave decay,
    1000 steps) and the 1024^2 multimode flow (10 steps), each on one thread
    and on all host threads, with the CPU model.  Minutes of CPU time."""
    import torch
    from paper_2510_04197_gb300 import inputs
    rows = []
    wave = inputs.wave_decay(64, 64, Ma=0.1, amp=1e-3)
    for threads in (1, None):
        v, el, used = oracle_mlups(64, 1000, 1, threads, fields=wave, P_kw=dict(Pr=0.71, gamma=1.4, mu=0.01))
        rows.append({"workload": "64^2 wave decay (config 1), 1000 steps", "threads": used, "mlups": v, "s": el})
        v, el, used = oracle_mlups(1024, 10, 1, threads)
        rows.append({"workload": "1024^2 periodic multimode, 10 steps", "threads": used, "mlups": v, "s": el})
    print(json.dumps({"cpu_table": rows, "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                      "torch_threads": torch.get_num_threads(), "kind": "oracle"}), flush=True)


def fp64_probe():
    """Measured FP64 FMA peak of this GPU (libdvbm_probe.so, CUDA events)."""
    import ctypes
    path = os.path.join(ROOT, "paper_2510_04197_gb300", "libdvbm_probe.so")
    try:
        L = ctypes.CDLL(path)
        L.dvbm_probe_fp64_fma.restype = ctypes.c_int
        tf, ms = ctypes.c_double(0), ctypes.c_double(0)
        rc = L.dvbm_probe_fp64_fma(5, ctypes.byref(tf), ctypes.byref(ms))
        if rc == 0:
            return {"tflops": tf.value, "best_ms": ms.value,
                    "how": "dvbm_probe_fp64_fma: 8 independent FMA chains x 4096 per thread, 8 x 256 threads per SM, "
                           "best of 5 launches, CUDA events"}
    except OSError:
        pass
    return None


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle on the host cores (rank 0 only)."""
    if rank != 0:
        return
    N = args.cpu_sample
    steps = args.steps
    cb = cpu_baseline(N, steps, warmup=max(1, args.warmup))
    line = {"metric": "MLUPS", "value": cb["value"], "unit": "MLUPS", "n_gpus": args.gpus, "steps": steps,
            "warmup": args.warmup, "ms_per_step": N * N / cb["value"] / 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.size, world, args.layout), "impl": "reference", "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def adjoint_ratio(dvbm, inputs, torch, N=512, nsteps=200):
    """Adjoint workload: N^2 periodic FP64, multimode rms Ma 0.3 (seed 0),
    Pr 0.71, gamma 1.4, mu 1e-3, nsteps steps, loss 1/(2N^2) sum[(rho - rho_t)^2
    + (T - T_t)^2] against the same flow from seed 1 after nsteps steps;
    checkpoints every ceil(sqrt(nsteps)).  ``ratio`` = the time of
    dvbm_adjoint (segment recompute + adjoint steps) over nsteps plain forward
    steps (CUDA events on an unrecorded context, after warm-up); the recorded
    forward run (init, checkpoint copies, moments to the host) is timed beside
    it."""
    import math as _m
    every = int(_m.ceil(_m.sqrt(nsteps)))
    tgt = inputs.multimode(N, seed=1, rms_Ma=0.3)
    st = dvbm.Simulation(N, N, 0.71, 1.4, 1e-3, check_every=-1)
    st.init(*(torch.tensor(a) for a in (tgt.rho, tgt.ux, tgt.uy, tgt.T)))
    st.step(nsteps)
    mt = st.moments()
    dt = st.dt
    st.close()
    F = inputs.multimode(N, seed=0, rms_Ma=0.3)
    fields = [torch.tensor(a, device="cuda") for a in (F.rho, F.ux, F.uy, F.T)]
    # plain forward steps: the denominator of the ratio
    plain = dvbm.Simulation(N, N, 0.71, 1.4, 1e-3, check_every=-1, dt=dt)
    plain.init(*fields)
    plain.step(5)
    torch.cuda.synchronize()
    fwd_ms, _ = timed_steps(plain, nsteps, torch.cuda.current_stream())
    plain.close()
    out = {}
    for rep in range(2):  # first repetition warms up allocations
        sim = dvbm.Simulation(N, N, 0.71, 1.4, 1e-3, check_every=-1, dt=dt)
        sim.record(every)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.init(*fields)
        sim.step(nsteps)
        m = sim.moments()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        n2 = N * N
        g = sim.adjoint((m["rho"] - mt["rho"]) / n2, (m["T"] - mt["T"]) / n2)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        # the stepwise pass a band of a decomposed grid runs (branches derived
        # from the states), on the same recording, one band: no neighbours
        gs = sim.adjoint_stepwise((m["rho"] - mt["rho"]) / n2, (m["T"] - mt["T"]) / n2)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        sim.close()
        out = {"workload": f"adjoint {N}x{N} periodic multimode rms Ma 0.3, {nsteps} FP64 steps, "
                           f"checkpoints every {every}",
               "t_forward_steps_ms": fwd_ms, "t_adjoint_ms": (t2 - t1) * 1e3,
               "ratio": (t2 - t1) * 1e3 / fwd_ms,
               "what": "t_adjoint / t_forward_steps: dvbm_adjoint (recompute + adjoint steps, wall clock) over "
                       "the same number of plain forward steps (CUDA events)",
               "t_recorded_forward_ms": (t1 - t0) * 1e3, "ratio_to_recorded_forward": (t2 - t1) / (t1 - t0),
               "stepwise": {"t_ms": (t3 - t2) * 1e3, "ratio": (t3 - t2) * 1e3 / fwd_ms,
                            "max_rel_diff": max(float((gs[k] - g[k]).abs().max() / g[k].abs().max())
                                                for k in ("rho0", "ux0", "uy0", "T0")),
                            "what": "dvbm_adjoint_begin/advance/finish on the same recording (the pass a band "
                                    "of a slab-decomposed grid runs), wall clock"},
               "grad_norms": {k: float(g[k].norm()) for k in ("rho0", "ux0", "uy0", "T0")},
               "dL_dparams": [g["mu"], g["Pr"], g["gamma"]]}
    return out


def timed_steps(sim, K, stream):
    """Time K single steps with CUDA events on the library's stream; returns
    (total ms, list of per-step ms)."""
    import torch
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    evs[0].record(stream)
    for i in range(K):
        sim.step(1)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    per = [evs[i].elapsed_time(evs[i + 1]) for i in range(K)]
    return evs[0].elapsed_time(evs[K]), per


def run_sweep(args):
    """Throughput sweep of the periodic multimode workload: N^2 for N in
    {1024, 2048, 4096}, rms Ma in {0.3, 0.6, 1.2}, FP64 and FP32-deviation
    storage; --steps timed steps (default 500 here) after --warmup.  A run
    that trips the instability flag is reported with the step count reached
    (the static lattices have a Mach limit)."""
    import torch
    from paper_2510_04197_gb300 import dvbm, inputs
    steps = args.steps if args.steps != 20 else 500
    stream = torch.cuda.current_stream()
    rows = []
    for N in (1024, 2048, 4096):
        for ma in (0.3, 0.6, 1.2):
            F = inputs.multimode(N, seed=0, rms_Ma=ma)
            fields = [torch.tensor(a) for a in (F.rho, F.ux, F.uy, F.T)]
            for storage in ("fp64", "fp32dev"):
                row = {"grid": N, "rms_Ma": ma, "storage": storage}
                sim = dvbm.Simulation(N, N, 0.71, 1.4, 5e-5, storage=1 if storage == "fp32dev" else 0,
                                      check_every=-1)
                try:
                    sim.init(*fields)
                    sim.step(args.warmup)
                    torch.cuda.synchronize()
                    total_ms, _ = timed_steps(sim, steps, stream)
                    sim.totals()  # raises if the run went unstable
                    row.update({"mlups": N * N * steps / (total_ms * 1e-3) / 1e6, "steps": steps,
                                "ms_per_step": total_ms / steps})
                except Exception as e:  # instability flag or bad state
                    row.update({"unstable": str(e).splitlines()[0][:160], "steps_reached": sim.steps})
                sim.close()
                rows.append(row)
                torch.cuda.empty_cache()
    print(json.dumps({"sweep": rows, "workload": "periodic multimode, Pr 0.71, gamma 1.4, mu 5e-5, CFL 0.01",
                      "unit": "MLUPS"}), flush=True)


def main():
    args = parse()
    if args.sweep:
        return run_sweep(args)
    if args.cpu_table:
        return cpu_table()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    from paper_2510_04197_gb300 import dvbm, inputs

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist:
            dist.barrier()

    N = args.size
    slabs = world > 1 and args.layout == "slabs"
    # slabs: every band holds the same flow, so the y-periodic global field is continuous across bands
    F = inputs.multimode(N, seed=0 if slabs else rank, rms_Ma=0.3)
    fields = [torch.tensor(a) for a in (F.rho, F.ux, F.uy, F.T)]
    stream = torch.cuda.current_stream()
    peaks, peak_kind = load_peaks()
    results = {}
    clocks = None
    variants = ["fp64"] + ([] if args.no_fp32dev else ["fp32dev"]) + ([] if args.no_d2q16 else ["d2q16"])
    for storage in variants:
        kw = dict(storage=1 if storage == "fp32dev" else 0, check_every=-1,
                  lattice=dvbm.D2Q16_SPLIT_I if storage == "d2q16" else dvbm.D2Q25_SPLIT_II)
        if slabs:
            from paper_2510_04197_gb300 import slab as SL
            sim = SL.RankSlab(dist, N, N, 0.71, 1.4, 5e-5, **kw)
        else:
            sim = dvbm.Simulation(N, N, 0.71, 1.4, 5e-5, **kw)
        sim.init(*fields)
        tot0 = sim.totals()  # outside the timed region: the conservation drift of the whole run
        sim.step(args.warmup)
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if storage == "fp64" else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        barrier()
        torch.cuda.synchronize()
        total_ms, per = timed_steps(sim, args.steps, stream)
        torch.cuda.synchronize()
        barrier()
        if sampler:
            clocks = sampler.stop()
        tmax = max_over_ranks(total_ms, dist, "cuda")
        mlups = whole_job_mlups(N * N, args.steps, world, tmax * 1e-3)
        tot = sim.totals()  # also raises if the run went unstable
        results[storage] = {"mlups": mlups, "ms_per_step": tmax / args.steps,
                            "kernel_ms": statistics.mean(per), "totals": tot,
                            "drift": conservation_drift(tot0, tot, args.warmup + args.steps)}
        sim.close()
        del sim
        torch.cuda.empty_cache()

    # the paper's shock--vortex case G grid (Sec. III.F: 1680 x 1440 over
    # [0, 28] x [0, 24], zero-gradient x, periodic y) as a second throughput
    # workload, both storage forms
    workloads = {}
    if not args.no_workloads:
        sv = inputs.shock_vortex_case("G")
        sf = [torch.tensor(a) for a in (sv.fields.rho, sv.fields.ux, sv.fields.uy, sv.fields.T)]
        bcs = [dvbm.ZEROGRAD, dvbm.ZEROGRAD, dvbm.PERIODIC, dvbm.PERIODIC]
        nx, ny = sv.fields.rho.shape[1], sv.fields.rho.shape[0]
        wl = {"workload": "shock-vortex case G (Ma_s 1.29, Ma_v 0.39, Re_v 800, Pr 0.75), 1680x1440 over 28x24, "
                          "zero-gradient x, periodic y, CFL 0.01"}
        for storage in ("fp64", "fp32dev"):
            sim = dvbm.Simulation(nx, ny, 0.75, 1.4, sv.mu, bcs=bcs, storage=1 if storage == "fp32dev" else 0,
                                  Lx=sv.fields.Lx, Ly=sv.fields.Ly, cfl=0.01, check_every=-1)
            sim.init(*sf)
            sim.step(args.warmup)
            torch.cuda.synchronize()
            barrier()
            total_ms, _ = timed_steps(sim, args.steps, stream)
            torch.cuda.synchronize()
            sim.totals()  # raises if the run went unstable
            wl[storage] = {"value": nx * ny * args.steps / (total_ms * 1e-3) / 1e6, "unit": "MLUPS",
                           "ms_per_step": total_ms / args.steps}
            sim.close()
        workloads["shock_vortex_G"] = wl
        torch.cuda.empty_cache()

    # end-to-end through the public API with host (pinned) buffers:
    # host fields -> dvbm_init -> K steps -> moments back to host
    e2e = None
    if not args.no_e2e:
        pin = [t.pin_memory() for t in fields]
        outs = {k: torch.empty((N, N), dtype=torch.float64).pin_memory() for k in ("rho", "ux", "uy", "T")}
        sim = dvbm.Simulation(N, N, 0.71, 1.4, 5e-5, storage=0, check_every=-1)
        sim.init_host(*[p.numpy() for p in pin])
        sim.step(1)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        sim.init_host(*[p.numpy() for p in pin])
        sim.step(args.steps)
        import ctypes
        st = dvbm.lib().dvbm_moments(sim._h, *[ctypes.c_void_p(outs[k].data_ptr()) for k in ("rho", "ux", "uy", "T")], 0)
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        assert st == 0
        e2e = {"value": whole_job_mlups(N * N, args.steps, world, el), "unit": "MLUPS",
               "h2d_bytes_per_step": 4 * 8 * N * N / args.steps, "d2h_bytes_per_step": 4 * 8 * N * N / args.steps,
               "note": "init from host fields + K steps + moments to host, per-step bytes = total / K"}
        sim.close()

    if rank != 0:
        return
    r64 = results["fp64"]
    # dominant kernel: the FP64 step; HBM roofline of its algorithmic bytes
    # (800 B per cell update: 50 populations read and written)
    hbm_peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    ach_gbs = BYTES_PER_CELL["fp64"] * N * N / (r64["kernel_ms"] * 1e-3) / 1e9
    tr = profile_traffic("k_step_fp64")
    roofline = {"bound": "hbm", "achieved": ach_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach_gbs / hbm_peak, "frac_of_8tbs": ach_gbs / NOMINAL_HBM_GBS,
                "traffic": (tr["dram_bytes_per_cell"] * N * N if tr else None),
                "kernel": "k_step<double> (FP64 storage, D2Q25 split II)",
                "what": "algorithmic 800 B per cell update x cells / step-kernel time (CUDA events); peak = "
                        + ("MEASURED_PEAKS.json hbm_gbs (of measured)" if peak_kind == "measured"
                           else "fallback 6.8 TB/s (of fallback)")}
    # the second ceiling on GB300: the FP64 pipe, against the measured FMA peak
    probe = fp64_probe()
    fp64_ops = tr.get("fp64_flops_per_cell") if tr else None
    roofline_fp64 = {"bound": "fp64", "unit": "TFLOP/s", "peak": probe["tflops"] if probe else NOMINAL_FP64_TFLOPS,
                     "peak_kind": "measured (dvbm_probe_fp64_fma)" if probe else "nominal (152 SMs x 2 x 2.07 GHz x 2)",
                     "probe": probe, "achieved": None, "frac": None}
    if fp64_ops:
        ach_tf = fp64_ops * N * N / (r64["kernel_ms"] * 1e-3) / 1e12
        roofline_fp64.update({"achieved": ach_tf, "frac": ach_tf / roofline_fp64["peak"],
                              "what": "executed FP64 flops per cell (ncu instruction mix of the profiled sources, "
                                      "FMA = 2) x cells / step-kernel time"})
        if tr.get("thread_inst_per_cell"):
            ach_is = tr["thread_inst_per_cell"] / 32.0 * N * N / (r64["kernel_ms"] * 1e-3) / 1e9
            roofline_fp64["issue"] = {"achieved": ach_is, "peak": NOMINAL_ISSUE_GWARPINST,
                                      "unit": "G warp-instructions/s", "frac": ach_is / NOMINAL_ISSUE_GWARPINST,
                                      "what": "all executed instructions (ncu) per cell / 32 x cells / step-kernel "
                                              "time; peak = 152 SMs x 4 schedulers x 2.07 GHz"}
    line = {"metric": "MLUPS", "value": r64["mlups"], "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r64["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(N, world, args.layout),
            "roofline": roofline, "roofline_fp64": roofline_fp64, "clocks": clocks,
            "gpu_launches": (4 if slabs else 2) * args.steps,
            "kernel_ms_per_step": r64["kernel_ms"], "conservation_drift": r64["drift"]}
    if "fp32dev" in results:
        r32 = results["fp32dev"]
        g32 = BYTES_PER_CELL["fp32dev"] * N * N / (r32["kernel_ms"] * 1e-3) / 1e9
        line["fp32dev"] = {"value": r32["mlups"], "unit": "MLUPS", "ms_per_step": r32["ms_per_step"],
                           "dtype": "f32 storage / f64 moments+equilibria", "conservation_drift": r32["drift"],
                           "roofline_hbm": {"bound": "hbm", "achieved": g32, "peak": hbm_peak, "unit": "GB/s",
                                            "frac": g32 / hbm_peak, "frac_of_8tbs": g32 / NOMINAL_HBM_GBS}}
        t32 = profile_traffic("k_step_fp32dev")
        line["fp32dev"]["roofline_hbm"]["traffic"] = t32["dram_bytes_per_cell"] * N * N if t32 else None
    if "d2q16" in results:
        r16 = results["d2q16"]
        g16 = BYTES_PER_CELL["d2q16"] * N * N / (r16["kernel_ms"] * 1e-3) / 1e9
        line["d2q16_split_I"] = {"value": r16["mlups"], "unit": "MLUPS", "ms_per_step": r16["ms_per_step"],
                                 "dtype": "f64", "workload": "same flow, total-energy split (I) on D2Q16",
                                 "conservation_drift": r16["drift"],
                                 "roofline_hbm": {"bound": "hbm", "achieved": g16, "peak": hbm_peak, "unit": "GB/s",
                                                  "frac": g16 / hbm_peak, "frac_of_8tbs": g16 / NOMINAL_HBM_GBS}}
        t16 = profile_traffic("k_step16")
        line["d2q16_split_I"]["roofline_hbm"]["traffic"] = t16["dram_bytes_per_cell"] * N * N if t16 else None
    line["e2e"] = e2e
    if workloads:
        line["workloads"] = workloads
    if not args.no_adjoint:
        line["adjoint"] = adjoint_ratio(dvbm, inputs, torch)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_sample)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
