#!/usr/bin/env python3
"""Throughput of the fused free-energy lattice Boltzmann step on GB300.

Workload: D3Q19, 128^3 periodic, one spherical drop R = 30 at the centre,
forcing scheme (Sec. VI), van der Waals a = 9/49, b = 2/21, T = 0.55,
kappa = 0.01, tau = 1.0 (synthetic drop, tanh profile of width 2).
A step is one time step of the whole lattice (one fused kernel launch).

Prints one JSON line: MLUPS (million lattice updates per second, whole job),
the HBM and ALU rooflines of the step kernel, an end-to-end number through
the C ABI with host buffers, the FP64 CPU oracle timed on a bounded sample,
and the time to steady state of a batched drop sweep against plain float64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--storage f16dev|bf16dev|f32|f64]
                  [--edge E] [--scheme forcing|equilibrium]
  python bench.py --impl reference ...     (the oracle, timed on the host cores)
Multi-GPU (N > 1, torchrun): independent replicas, one per GPU (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

A_VDW, B_VDW = 9.0 / 49.0, 2.0 / 21.0
WORKLOAD = dict(lattice="D3Q19", n=128, R=30.0, scheme="forcing", T=0.55, kappa=0.01, tau=1.0, width=2.0)
BYTES_POP = {"f64": (8, 8), "f32": (4, 4), "f16dev": (4, 2), "bf16dev": (4, 2)}   # (f_0, f_i) bytes


KERNEL_SOURCES = ["step3d.cuh", "step3d_pk.cuh", "kern_d3q19_pk.cu", "step_kernel.cuh", "storage.cuh", "lattice.cuh"]
# DRAM bytes (read + write) per launch of the D3Q19 forcing step kernel at
# 128^3, from ncu (dram__bytes_read.sum + dram__bytes_write.sum), keyed by the
# fingerprint of the kernel sources they were measured on and the storage.
# A changed kernel has a new fingerprint and reports traffic = null.
NCU_TRAFFIC = {
    ("412489fce235", "f16dev", 128): 142.85e6,   # 103.35 MB read + 39.50 MB written (pair kernel)
    ("412489fce235", "bf16dev", 128): 143.09e6,  # 103.39 MB read + 39.70 MB written (pair kernel)
    ("412489fce235", "f32", 128): 301.60e6,      # 188.75 MB read + 112.85 MB written (pair kernel, 2 CTAs per SM)
    ("412489fce235", "f64", 128): 637.11e6,      # 357.07 MB read + 280.05 MB written (tile kernel)
}

# Executed floating-point operations per lattice update of the step kernel,
# from ncu's per-opcode instruction counts of one launch divided by the sites
# (FFMA, DFMA, FADD2, FMUL2 = 2 flops, FFMA2 = 4; FADD, FMUL, FHADD, DADD,
# DMUL = 1), keyed like
# NCU_TRAFFIC.  They include the halo recomputation, so they are the work the
# FP units do, not an algorithmic minimum.
NCU_FLOPS = {
    # pair kernel: FFMA 10.8, FADD 64.3, FMUL 20.6, FADD2 36.6, FFMA2 43.9, FMUL2 29.9, FHADD 75.2 per site
    ("412489fce235", "f16dev", 128): 490.5,
    # float32 pair kernel: FFMA 10.3, FADD 61.5, FMUL 17.8, FADD2 64.8, FFMA2 43.5, FMUL2 29.6
    ("412489fce235", "f32", 128): 462.7,
    ("412489fce235", "f64", 128): 525.6,       # tile kernel: DFMA 129.0, DADD 197.4, DMUL 70.2
}
# FP64-pipe instructions per lattice update of the float64 step (DFMA, DADD,
# DMUL, DSETP, F2F): each occupies the pipe like one FMA, so their rate against
# half the FMA flop rate is the pipe's utilisation.
NCU_FP64_PIPE_OPS = {("412489fce235", "f64", 128): 401.7}


def alu_roofline(fp: str, storage: str, n: int, glups: float, fma: dict | None):
    """Executed flops per second of the step kernel against the GPU's measured
    FMA rate (lb_fma_peak; float64 units for float64 storage, float32 otherwise)."""
    flop = NCU_FLOPS.get((fp, storage, n))
    if flop is None or not fma:
        return None
    prec = "f64" if storage == "f64" else "f32"
    achieved = flop * glups * 1e9 / 1e12
    out = {"bound": "alu", "precision": prec, "flop_per_lu": flop, "achieved": achieved, "peak": fma[prec],
           "unit": "TFLOP/s", "frac": achieved / fma[prec],
           "peak_source": f"lb_fma_peak {prec} (measured in this run: FMA chains on every SM)"}
    ops = NCU_FP64_PIPE_OPS.get((fp, storage, n))
    if ops is not None:
        out["fp64_pipe_ops_per_lu"] = ops
        out["pipe_frac"] = ops * glups * 1e9 / (fma[prec] * 1e12 / 2)
    return out


def kernel_fingerprint() -> str:
    import hashlib
    h = hashlib.sha1()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_0710_5470_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def bytes_per_lu(storage: str, q: int = 19) -> int:
    """Algorithmic HBM bytes per lattice update of the reported roofline: one
    read and one write of every stored population plus one read and one write
    of the density, B = 2 Q s_f + 2 s_rho (s_rho = 4, or 8 for float64):
    88 B for 16-bit deviations (f_0 float32), 160 B float32, 320 B float64."""
    b0, bi = BYTES_POP[storage]
    s_rho = 8 if storage == "f64" else 4
    return 2 * (b0 + (q - 1) * bi) + 2 * s_rho


def bytes_moved_per_lu(storage: str, q: int = 19) -> int:
    """Bytes per lattice update this design moves: the populations once in and
    once out (the density is recomputed on chip and never stored): 80 B for
    16-bit deviations, 152 B float32, 304 B float64."""
    b0, bi = BYTES_POP[storage]
    return 2 * (b0 + (q - 1) * bi)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=4000)
    p.add_argument("--warmup", type=int, default=100)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--storage", default="f16dev", choices=list(BYTES_POP))
    p.add_argument("--edge", type=int, default=WORKLOAD["n"], help="lattice edge (default 128)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--no-steady", action="store_true")
    p.add_argument("--oracle-table", action="store_true",
                   help="only time the FP64 oracle on the paper-shaped workloads (one core, all cores) and exit")
    p.add_argument("--scheme", default="forcing", choices=["forcing", "equilibrium"],
                   help="collision scheme (the headline workload is the forcing scheme)")
    return p.parse_args()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.idx = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return self.parse(out)

    @staticmethod
    def parse(out: str) -> dict:
        """Median SM clock, maximum SM clock and the throttle reasons seen in
        nvidia-smi CSV lines of FIELDS (noheader, nounits)."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local, dist


def reduce_max(dist, value: float) -> float:
    if dist is None:
        return value
    import torch
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


def whole_job(dist, world: int, sites_per_rank: int, steps: int, ms_local: float):
    """Slowest rank's time (ms) and the whole-job MLUPS: every rank advances
    its own replica of sites_per_rank sites by `steps` steps."""
    ms = reduce_max(dist, ms_local)
    return ms, sites_per_rank * steps * world / (ms / 1e3) / 1e6


def oracle_sample(n_edge: int, steps: int, scheme: str = "forcing"):
    """FP64 oracle on an n_edge^3 periodic box holding the same drop scaled to
    the box (R = 30/128 of the edge): returns (MLUPS, seconds, sites*steps)."""
    from oracle import lb_oracle as O
    m = O.Model("D3Q19", A_VDW, B_VDW, WORKLOAD["T"], WORKLOAD["kappa"], WORKLOAD["tau"], scheme=scheme)
    rl, rg = O.coexistence(A_VDW, B_VDW, WORKLOAD["T"])
    R = WORKLOAD["R"] * n_edge / WORKLOAD["n"]
    rho0 = O.drop_density((n_edge,) * 3, [(n_edge / 2,) * 3], [R], rl, rg, WORKLOAD["width"])
    f = O.init_equilibrium(rho0, m)
    t0 = time.perf_counter()
    for _ in range(steps):
        f = O.step(f, m)
    dt = time.perf_counter() - t0
    lu = n_edge ** 3 * steps
    return lu / dt / 1e6, dt, lu


def cpu_model() -> str:
    """Name of the host CPU (lscpu's model name, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# oracle timing table: workload name -> (lattice, shape (nz, ny, nx), scheme, T, kappa, tau, drops, steps, warm-up)
ORACLE_TABLE = {
    "D2Q9 64^2, one drop R=16, equilibrium scheme, T=0.55, kappa=0.01, tau=1": ("D2Q9", (1, 64, 64), "equilibrium",
                                                                               0.55, 0.01, 1.0, "centre16", 200, 10),
    "D2Q9 512^2, drops of random_drops(0), forcing scheme, T=0.55, kappa=0.01, tau=0.8": (
        "D2Q9", (1, 512, 512), "forcing", 0.55, 0.01, 0.8, "random0", 20, 2),
    "D2Q9 512^2, drops of random_drops(0), equilibrium scheme, T=0.55, kappa=0.01, tau=0.8": (
        "D2Q9", (1, 512, 512), "equilibrium", 0.55, 0.01, 0.8, "random0", 20, 2),
    # the 128^3 workload scaled to 64^3 (R = 15): bounded host memory with one copy per core
    "D3Q19 64^3, one drop R=15, forcing scheme, T=0.55, kappa=0.01, tau=1": ("D3Q19", (64, 64, 64), "forcing",
                                                                             0.55, 0.01, 1.0, "centre15", 10, 1),
}


def _oracle_table_worker(job):
    """Time one oracle configuration (a value of ORACLE_TABLE; one process, one
    thread): warm-up steps, wait for the others, timed steps."""
    cfg, bar = job
    lat, shape, scheme, T, kappa, tau, drops, steps, warm = cfg
    from oracle import lb_oracle as O
    from paper_0710_5470_gb300 import inputs
    m = O.Model(lat, A_VDW, B_VDW, T, kappa, tau, scheme=scheme)
    rl, rg = O.coexistence(A_VDW, B_VDW, T)
    nz, ny, nx = shape
    if drops == "random0":
        centres, radii, _ = inputs.random_drops(0, (nx, ny))
    elif lat == "D2Q9":
        centres, radii = [(nx / 2, ny / 2)], [float(drops[6:])]
    else:
        centres, radii = [(nx / 2, ny / 2, nz / 2)], [float(drops[6:])]
    rho0 = O.drop_density(shape, centres, radii, rl, rg, 2.0)
    f = O.init_equilibrium(rho0, m)
    for _ in range(warm):
        f = O.step(f, m)
    if bar is not None:
        bar.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        f = O.step(f, m)
    dt = time.perf_counter() - t0
    return nx * ny * nz * steps / dt / 1e6


def oracle_table() -> dict:
    """The FP64 oracle's step rate (MLUPS) on the paper-shaped workloads, on one
    host core and on every host core at once (one single-threaded process per
    core, each on its own copy of the workload; the larger copies are bounded to
    a few steps each)."""
    import multiprocessing as mp
    procs = len(os.sched_getaffinity(0))
    keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in keep:
        os.environ[k] = "1"
    out = {"cpu": cpu_model(), "cores": procs, "rows": {}}
    try:
        ctx = mp.get_context("spawn")
        for name, cfg in ORACLE_TABLE.items():
            one = _oracle_table_worker((cfg, None))
            with ctx.Manager() as man:
                bar = man.Barrier(procs)
                with ctx.Pool(procs) as pool:
                    rates = pool.map(_oracle_table_worker, [(cfg, bar)] * procs)
            steps, warm = cfg[7], cfg[8]
            out["rows"][name] = {"one_core_mlups": one, "all_cores_mlups": float(sum(rates)),
                                 "cores": procs, "steps": steps, "warmup": warm}
    finally:
        for k, v in keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return out


def _oracle_worker(job):
    """One process of the all-core oracle run: `warmup` untimed steps, wait for
    the others, then time `steps` oracle steps on its own edge^3 drop box."""
    edge, steps, scheme, bar, warmup = job
    from oracle import lb_oracle as O
    m = O.Model("D3Q19", A_VDW, B_VDW, WORKLOAD["T"], WORKLOAD["kappa"], WORKLOAD["tau"], scheme=scheme)
    rl, rg = O.coexistence(A_VDW, B_VDW, WORKLOAD["T"])
    R = WORKLOAD["R"] * edge / WORKLOAD["n"]
    f = O.init_equilibrium(O.drop_density((edge,) * 3, [(edge / 2,) * 3], [R], rl, rg, WORKLOAD["width"]), m)
    for _ in range(warmup):
        f = O.step(f, m)
    bar.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        f = O.step(f, m)
    return time.perf_counter() - t0


def oracle_all_cores(edge: int, steps: int, scheme: str = "forcing", procs: int | None = None, warmup: int = 0):
    """The oracle on every host core at once: `procs` single-threaded processes
    (spawned), each stepping its own edge^3 box; returns (aggregate MLUPS,
    seconds of the slowest, processes)."""
    import multiprocessing as mp
    procs = procs or len(os.sched_getaffinity(0))
    keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in keep:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Manager() as man:
            bar = man.Barrier(procs)
            with ctx.Pool(procs) as pool:
                dts = pool.map(_oracle_worker, [(edge, steps, scheme, bar, warmup)] * procs)
    finally:
        for k, v in keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    dt = max(dts)
    return procs * edge ** 3 * steps / dt / 1e6, dt, procs


# ---------------------------------------------------------------- arms
def run_reference(args):
    world, rank, local, dist = dist_setup(args.gpus)
    if rank != 0:
        return
    # the oracle on every host core: one single-threaded process per core, each
    # stepping its own sub-box of the workload (the drop scaled to the box), the
    # box sized so that the whole run stays within about two minutes
    procs = max(1, len(os.sched_getaffinity(0)))
    budget = 120.0 / max(1, args.steps + args.warmup)
    rate = 0.25e6                                     # oracle LU/s per core, measured order of magnitude
    edge = int(max(8, min(args.edge, round((budget * rate) ** (1 / 3)))))
    if procs > 1:
        edge = min(edge, 64)                            # bounded host memory: one box per process
    try:
        mlups, dt, procs = oracle_all_cores(edge, args.steps, args.scheme, procs, warmup=args.warmup)
        cores = procs
    except Exception:                                   # no process support: one core
        mlups, dt, _ = oracle_sample(edge, args.steps, args.scheme)
        cores = 1
    sample = (f"{cores} single-threaded FP64 oracle processes (numpy) at once, each {args.steps} timed steps "
              f"after {args.warmup} on its own {edge}^3 box (the drop scaled to the box)")
    line = {"impl": "reference", "metric": f"MLUPS (D3Q19 128^3 free-energy LB step, {args.scheme} scheme)",
            "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"D3Q19 {WORKLOAD['n']}^3 drop R=30, {args.scheme} scheme, T=0.55, kappa=0.01, tau=1",
                       "sample_edge": edge},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu": cpu_model()},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_steps(ctx, stream, steps, dist=None):
    """CUDA-event time (ms) of exactly `steps` fused steps, one kernel launch
    each, run by one lb_step call on the context's stream (lb_step replays
    its captured graphs of 64 steps; they are captured in the warm-up when
    it is longer than 64 steps, else at the start of this call)."""
    import torch
    barrier(dist)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    ctx.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    return ev0.elapsed_time(ev1)


def make_ctx(lb, storage: str, n: int, stream, scheme: str = "forcing"):
    ctx = lb.Context(lb.D3Q19, (n, n, n), A_VDW, B_VDW, WORKLOAD["T"], WORKLOAD["kappa"], WORKLOAD["tau"],
                     scheme=lb.FORCING if scheme == "forcing" else lb.EQUILIBRIUM,
                     storage=lb.STORAGE_NAMES[storage], stream=stream.cuda_stream)
    R = WORKLOAD["R"] * n / WORKLOAD["n"]
    ctx.init_drops([(n / 2,) * 3], [R], WORKLOAD["width"])
    return ctx, R


BINARY = {"n": 2048, "R": 512.0, "A": -0.04, "B": 0.04, "kappa": 0.08, "Gamma": 1.0, "tau": 1.0, "tau_phi": 1.0}


def binary_block(lb, stream, peak, dist, world, warmup, cpu: bool):
    """D2Q9 binary fluid, one drop of phase +phi* (R = n/4, tanh profile of
    width w = sqrt(-2 kappa / A)) in -phi*, rho = 1: GLUPS of the fused step in
    float32 and float64 storage, both schemes, against the HBM roofline at the
    bytes it moves (18 populations read and written: 144 / 288 B per update)."""
    import numpy as np
    from paper_0710_5470_gb300 import binary as bin_runs
    b = BINARY
    n = b["n"]
    w = bin_runs.interface_width(b["A"], b["kappa"])
    phi0 = bin_runs.drop_phi(n, b["R"], b["A"], b["kappa"], b["B"])
    out = {"workload": f"D2Q9 {n}^2 periodic, one drop R={b['R']:g} of phi=+1 in phi=-1 (tanh, width "
                       f"{w:g}), rho=1, A={b['A']}, B={b['B']}, kappa={b['kappa']}, Gamma={b['Gamma']}, "
                       f"tau=tau_phi=1", "runs": {}}
    for scheme in ("forcing", "equilibrium"):
        for sname, st_code, bpl, steps in (("f32", lb.F32, 144, 400), ("f16dev", lb.F16DEV, 80, 400),
                                           ("f64", lb.F64, 288, 100)):
            ctx = lb.BinaryContext((n, n), b["A"], b["B"], b["kappa"], b["Gamma"], b["tau"], b["tau_phi"],
                                   scheme=lb.FORCING if scheme == "forcing" else lb.EQUILIBRIUM, storage=st_code,
                                   stream=stream.cuda_stream)
            ctx.init_fields(np.ones((n, n)), phi0)
            ctx.step(max(warmup, 64))
            ctx.synchronize()
            ms = reduce_max(dist, time_steps(ctx, stream, steps, dist))
            stt = ctx.stats()
            ctx.close()
            t = ms / steps / 1e3
            ach = bpl * n * n / t / 1e9
            out["runs"][f"{scheme}_{sname}"] = {
                "value": n * n * steps * world / (ms / 1e3) / 1e6, "unit": "MLUPS", "steps": steps,
                "ms_per_step": ms / steps,
                "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                             "bytes_per_lu": bpl},
                "max_v": stt["max_v"], "status": stt["status"]}
    # D3Q19: 128^3, one drop R = 32; two launches per step (the phi pass and the
    # fused step), algorithmic bytes the 38 populations read and written
    n3 = 128
    phi3 = bin_runs.drop_phi(n3, 32.0, b["A"], b["kappa"], b["B"], dim=3)
    out["workload_3d"] = (f"D3Q19 {n3}^3 periodic, one drop R=32 of phi=+1 in phi=-1 (tanh, width {w:g}), "
                          f"rho=1, the same parameters")
    for scheme in ("forcing", "equilibrium"):
        for sname, st_code, bpl, steps in (("f32", lb.F32, 304, 200), ("f64", lb.F64, 608, 40)):
            ctx = lb.BinaryContext((n3, n3, n3), b["A"], b["B"], b["kappa"], b["Gamma"], b["tau"], b["tau_phi"],
                                   scheme=lb.FORCING if scheme == "forcing" else lb.EQUILIBRIUM, storage=st_code,
                                   stream=stream.cuda_stream)
            ctx.init_fields(np.ones((n3, n3, n3)), phi3)
            ctx.step(max(warmup, 64) if sname == "f32" else 8)
            ctx.synchronize()
            ms = reduce_max(dist, time_steps(ctx, stream, steps, dist))
            stt = ctx.stats()
            ctx.close()
            t = ms / steps / 1e3
            ach = bpl * n3 ** 3 / t / 1e9
            out["runs"][f"d3q19_{scheme}_{sname}"] = {
                "value": n3 ** 3 * steps * world / (ms / 1e3) / 1e6, "unit": "MLUPS", "steps": steps,
                "ms_per_step": ms / steps,
                "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                             "bytes_per_lu": bpl, "note": "the phi pass adds 80 B (float32) per update"},
                "max_v": stt["max_v"], "status": stt["status"]}
    if cpu:
        from oracle import binary_oracle as BO
        m = BO.BinaryModel("D2Q9", b["A"], b["B"], b["kappa"], b["Gamma"], b["tau"], b["tau_phi"], scheme="forcing")
        ns = 512
        ys, xs = np.meshgrid(np.arange(ns, dtype=np.float64), np.arange(ns, dtype=np.float64), indexing="ij")
        ds = np.hypot(xs - ns / 2, ys - ns / 2)
        f, g = BO.init_equilibrium(np.ones((1, ns, ns)), (-1.0 + (1 + np.tanh((ns / 4 - ds) / w)))[None], m)
        t0 = time.perf_counter()
        BO.run(f, g, m, 3)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": ns * ns * 3 / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                               "sample": f"3 FP64 binary-oracle steps (numpy, one thread), forcing scheme, the "
                                         f"workload scaled to {ns}^2 ({dt:.1f} s)"}
    return out


def run_native(args):
    import numpy as np
    import torch

    world, rank, local, dist = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    from paper_0710_5470_gb300 import build, lb
    if rank == 0:
        build.build()
    barrier(dist)
    if rank != 0:
        build.build()
    lb.load_library()
    n = args.edge
    sites = n ** 3
    stream = torch.cuda.current_stream()
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    fp = kernel_fingerprint()

    ctx, R = make_ctx(lb, args.storage, n, stream, args.scheme)
    kinfo = ctx.kernel_info()
    ctx.step(args.warmup)
    ctx.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms_local = time_steps(ctx, stream, args.steps, dist)
    clk = clocks.stop()
    ctx.synchronize()
    st = ctx.stats()
    ms, mlups = whole_job(dist, world, sites, args.steps, ms_local)

    # roofline of the fused step kernel (the only kernel in the timed region):
    # algorithmic bytes per launch / average launch duration
    bpl = bytes_per_lu(args.storage)
    t_launch = ms_local / args.steps / 1e3
    achieved = bpl * sites / t_launch / 1e9
    # the ncu tables hold the forcing-scheme kernel
    forcing = args.scheme == "forcing"
    traffic = NCU_TRAFFIC.get((fp, args.storage, n)) if forcing else None
    # FMA rates of this GPU (float64 and float32), best of three short launches
    fma = {"f64": max(lb.fma_peak(0) for _ in range(3)), "f32": max(lb.fma_peak(1) for _ in range(3))}
    alu = alu_roofline(fp, args.storage, n, sites / t_launch / 1e9, fma) if forcing else None

    # end to end through the C ABI with host buffers (pinned): upload the initial
    # density, run the steps, download rho and u
    e2e = None
    if not args.no_e2e:
        rl, rg = ctx.coexistence()
        rho_h = torch.empty(sites, dtype=torch.float64, pin_memory=True).numpy()
        z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64),) * 3, indexing="ij")
        d = np.sqrt((x - n / 2) ** 2 + (y - n / 2) ** 2 + (z - n / 2) ** 2)
        rho_h[:] = (rg + (rl - rg) * 0.5 * (1 + np.tanh((R - d) / WORKLOAD["width"]))).reshape(-1)
        out_rho = torch.empty(sites, dtype=torch.float64, pin_memory=True).numpy()
        out_u = torch.empty(3 * sites, dtype=torch.float64, pin_memory=True).numpy()
        barrier(dist)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.init_fields(rho_h)
        ctx.step(args.steps)
        ctx.fields_into(out_rho, out_u)
        dt = reduce_max(dist, time.perf_counter() - t0)
        e2e = {"value": sites * args.steps * world / dt / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": sites * 8 / args.steps, "d2h_bytes_per_step": sites * 8 * 4 / args.steps,
               "note": "init from a host density field, K steps, rho and u back to the host"}
    ctx.close()

    variants = {}
    if not args.no_variants:
        for sname in BYTES_POP:
            if sname == args.storage:
                continue
            vctx, _ = make_ctx(lb, sname, n, stream, args.scheme)
            vsteps = max(1, args.steps // (20 if sname == "f64" else 1))
            vctx.step(min(args.warmup, 5) if sname == "f64" else args.warmup)
            vctx.synchronize()
            vms = reduce_max(dist, time_steps(vctx, stream, vsteps, dist))
            vst = vctx.stats()
            vctx.close()
            vb = bytes_per_lu(sname)
            vach = vb * sites / (vms / vsteps / 1e3) / 1e9
            variants[sname] = {"value": sites * vsteps * world / (vms / 1e3) / 1e6, "steps": vsteps,
                               "ms_per_step": vms / vsteps,
                               "roofline": {"bound": "hbm", "achieved": vach, "peak": peak, "unit": "GB/s",
                                            "frac": vach / peak, "bytes_per_lu": vb,
                                            "traffic": NCU_TRAFFIC.get((fp, sname, n)) if forcing else None},
                               "alu_roofline": alu_roofline(fp, sname, n, sites / (vms / vsteps / 1e3) / 1e9,
                                                            fma) if forcing else None,
                               "max_v": vst["max_v"]}

    # the same lattice with the equilibrium scheme (Secs. II-V: no body force),
    # the storage formats of 32-bit arithmetic, for context beside the forcing line
    other_scheme = {}
    if not args.no_variants and forcing:
        for sname in ("f16dev", "f32"):
            ectx, _ = make_ctx(lb, sname, n, stream, "equilibrium")
            ectx.step(args.warmup)
            ectx.synchronize()
            esteps = args.steps
            ems = reduce_max(dist, time_steps(ectx, stream, esteps, dist))
            est = ectx.stats()
            einfo = ectx.kernel_info()
            ectx.close()
            eb = bytes_per_lu(sname)
            each = eb * sites / (ems / esteps / 1e3) / 1e9
            other_scheme[sname] = {"value": sites * esteps * world / (ems / 1e3) / 1e6, "steps": esteps,
                                   "ms_per_step": ems / esteps, "kernel": einfo["form"],
                                   "roofline": {"bound": "hbm", "achieved": each, "peak": peak, "unit": "GB/s",
                                                "frac": each / peak, "bytes_per_lu": eb},
                                   "max_u": est["max_u"]}

    # the binary-fluid model (the paper's construction carried over to an order
    # parameter, Sec. I): D2Q9 fused step, both storage formats, forcing scheme
    binary = None
    if not args.no_variants:
        binary = binary_block(lb, stream, peak, dist, world, args.warmup, not args.no_cpu_baseline and rank == 0)

    # time to steady state (second half of the metric): plain float64, one
    # instance per launch, to max|u(t) - u(t - 100)| < 1e-10, against one batch
    # in fp16-deviation storage stopped by its own self-contained test (max|u|
    # and bulk densities settled; no steady values known in advance); accuracy
    # of the fast steady states afterwards against the float64 ones
    tts = None
    if rank == 0 and world == 1 and not args.no_steady:
        from paper_0710_5470_gb300 import steady
        ex = steady.experiment_self(count=16, seed=0, arms=("f16dev",))
        fa = ex["batch_f16dev_self"]
        pl = ex["plain_f64_tol"]
        tts = {"workload": "first 16 instances of the D2Q9 drop sweep seed 0 (side 64-384, T 0.50-0.56, "
                           "kappa 0.002-0.03, tau 0.6-1.5, one centred drop, forcing scheme)",
               "plain": "float64, one instance per batch, tanh start, to max|u(t) - u(t-100)| < 1e-10",
               "fast": "one batch, fp16-deviation storage, CUDA-graph replay, autotuned tile, stopped when "
                       "max|u| changes by < 5e-4 of itself and max/min rho by < 1e-5 per 100 steps for 10 "
                       "consecutive checks (lb_batch_set_self_test; no reference values)",
               "plain_f64_s": pl["seconds"], "fast_s": fa["seconds"], "speedup": pl["seconds"] / fa["seconds"],
               "converged": {"plain": pl["converged"], "fast": fa["converged"]},
               "mean_steps": {"plain": pl["mean_steps"], "fast": fa["mean_steps"]},
               "accuracy_fast": {"max_u_rel_err_max": fa.get("max_u_rel_err_max"),
                                 "rho_max_err_max": fa.get("rho_max_err_max"),
                                 "rho_min_err_max": fa.get("rho_min_err_max"),
                                 "within_5pct_of_f64_max_u": f"{fa['within_5pct']} of {fa['compared']}"}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        edge = n
        v, dt, lu = oracle_sample(edge, 5, args.scheme)
        model = cpu_model()
        cpu = {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle", "cpu": model,
               "sample": f"5 FP64 oracle steps (numpy, one thread) on the full {edge}^3 drop workload ({dt:.1f} s)"}
        try:
            va, dta, procs = oracle_all_cores(64, 4, args.scheme)
            cpu["all_cores"] = {"value": va, "unit": "MLUPS", "cores": procs, "kind": "oracle", "cpu": model,
                                "sample": f"{procs} single-threaded oracle processes at once, each 4 FP64 steps "
                                          f"of its own 64^3 drop box (the workload scaled to 64^3; "
                                          f"slowest {dta:.1f} s)"}
        except Exception as e:                                  # a host without process support
            cpu["all_cores"] = {"unavailable": repr(e)}

    if rank == 0:
        line = {
            "metric": f"MLUPS (D3Q19 {n}^3 free-energy LB step, {args.scheme} scheme)",
            "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.storage != "f64" else "f64", "data": "synthetic",
            "config": {"workload": f"D3Q19 {n}^3 periodic, one drop R={R:g}, {args.scheme} scheme, T=0.55, "
                                   f"kappa=0.01, tau=1.0", "storage": args.storage,
                       "l2": "inputs larger than L2: the two population buffers exceed the 126 MB L2",
                       "parallelism": f"{world} independent replica(s)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "bytes_per_lu": bpl,
                         "bytes_moved_per_lu": bytes_moved_per_lu(args.storage),
                         "frac_of_moved": achieved * bytes_moved_per_lu(args.storage) / bpl / peak,
                         "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback",
                         "kernel_fingerprint": fp},
            "alu_roofline": alu,
            "kernel": kinfo,
            "fma_peak_tflops": fma,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": clk,
            "variants": variants,
            "equilibrium_scheme": other_scheme or None,
            "binary_fluid": binary,
            "time_to_steady": tts,
            "check": {"max_v": st["max_v"], "mass": st["mass"], "status": st["status"]},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.oracle_table:
        print(json.dumps(oracle_table()), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
