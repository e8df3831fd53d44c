"""Benchmark: MLUPS and fraction of the HBM roofline of the fused stream-collide step on GB300.

Workload (one benchmark step = one pass of the whole hot path over one synthetic input):
  2D periodic D2Q5 grid of 2048 x 2048 cells, FP32 storage and arithmetic, tau = 0.6, initial
  field = Gaussian pulse (amplitude 1e-3, width 32 cells) + 8 density plane waves (amplitude
  1e-4, wavelength 16-256 cells), seed 2;  init_fields (equilibrium of the fields) -> 1000 time
  steps -> per-cell moments -> FP64 global sums.
value   = cells * 1000 * K / (sum of the K device-timed steps), in MLUPS (10^6 lattice updates/s).
e2e     = the same through the C ABI with pinned host buffers: fields copied in and moments copied
          out inside the timed region.
Extra forms (not part of the timed value): 3D D3Q7 384^3 with FP32/FP16/BF16 storage against the
FP64 run (MLUPS and relative L2 of rho').

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-forms]
With N > 1 (torchrun, one process per GPU) every rank runs an independent replica of the
workload ("replicas only": the single-domain path has no exchange step on one box).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
NX = 2048
NSTEPS = 1000
TAU = 0.6
SET = "D2Q5"
STORAGE = "f32"
BYTES_PER_LUP = 2 * 5 * 4  # read + write of q = 5 FP32 populations (algorithmic)
L2_FLUSH_BYTES = 512 << 20
NOMINAL_HBM_GBS = 8000.0  # HBM3e nominal bandwidth of the part (the measured copy peak is the denominator of frac)
WORKLOAD = "2D D2Q5 periodic 2048x2048, FP32, tau=0.6, pulse+8 plane waves, 1000 steps/job"
METRIC = "MLUPS (2D D2Q5 FP32 stream-collide job) and fraction of HBM roofline"
# ncu summary of the stream-collide kernel the benchmark runs, by time steps fused per launch
PROFILES = {k: os.path.join(ROOT, "profiles", f"stream_collide_{k}step_d2q5_f32_2048x2048.md") for k in (1, 2, 3, 4)}
KERNEL_NAMES = {1: "k_stream_collide<D2Q5,float,V=4,periodic>", 2: "k_stream_collide_2step<D2Q5,float>",
                3: "k_stream_collide_kstep<D2Q5,K=3,float>", 4: "k_stream_collide_kstep<D2Q5,K=4,float>"}
KERNEL_SOURCES = ["paper_1601_08103_gb300/csrc/kernels.cuh", "paper_1601_08103_gb300/csrc/step_launch.cuh",
                  "paper_1601_08103_gb300/csrc/velsets.cuh"]


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(steps_per_launch: int):
    """DRAM bytes per stream-collide launch from the committed ncu summary of the kernel that
    fuses this many steps, or None if the summary is missing or was taken on different kernel
    sources."""
    path = PROFILES.get(steps_per_launch)
    if not path or not os.path.exists(path):
        return None
    txt = open(path).read()
    sha = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    tr = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not sha or not tr or sha.group(1) != kernel_source_sha():
        return None
    return float(tr.group(1))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, path: str | None = None):
        """Samples go to `path` (kept), or to a temporary file removed after stop()."""
        self.index = index
        self.proc = None
        self.keep = path is not None
        if path is None:
            fd, path = tempfile.mkstemp(prefix=f"lee_clocks_rank{index}_", suffix=".csv")
            os.close(fd)
        self.path = path

    def start(self):
        try:
            if os.path.dirname(self.path):
                os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # nvidia-smi takes a moment to start: wait (at most 3 s) for its first line so that the
        # samples cover the timed region
        t0 = time.time()
        while time.time() - t0 < 3.0 and self.proc.poll() is None:
            self.f.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            lines = f.readlines()
        if not self.keep:
            os.unlink(self.path)
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = np.array([r[0] for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[2][k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(r[1] for r in rows)), "reasons": reasons,
                "samples": len(rows)}


def dist_setup(ngpus: int):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def max_over_ranks(value: float, world: int) -> float:
    """Maximum of a per-rank float over all ranks (the job is as slow as its slowest rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def bench_config(world: int) -> dict:
    """The workload description both arms print (identical, so the two lines compare)."""
    return {"workload": WORKLOAD, "cells": NX * NX, "lbm_steps_per_job": NSTEPS, "velset": SET, "tau": TAU,
            "storage": STORAGE, "parallelism": f"replicas{world}",
            "l2": "512 MiB write between timed steps; ping-pong working set 168 MB > 129 MB L2"}


def run_ours(args, rank, world, local):
    import torch

    import paper_1601_08103_gb300 as lee
    from paper_1601_08103_gb300 import inputs

    lee.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    cells = NX * NX
    rho, u, th = inputs.config_2d(NX, seed=2)
    rho_d = torch.from_numpy(rho).to(dev)
    u_d = torch.from_numpy(u).to(dev)
    th_d = torch.from_numpy(th).to(dev)
    mom_d = torch.empty((4, cells), dtype=torch.float64, device=dev)
    red_d = torch.empty(8, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sv = lee.Solver(SET, (NX, NX, 1), TAU, storage=STORAGE, stream=stream)

    # steps per stream-collide launch: 4 for this periodic 2D FP32 grid (four fused time steps
    # per launch, the intermediate states in shared memory), 1 for the one-step kernel.  A job of
    # NSTEPS steps is NSTEPS // spl fused launches and NSTEPS % spl single steps; every launch reads
    # and writes the whole state once, so each moves the same algorithmic bytes.
    spl = max(sv.steps_per_launch, 1)
    step_launches = NSTEPS // spl + NSTEPS % spl
    launches_per_step = 1 + step_launches + 1 + 2  # init, steps, moments, reduce (partial + final)

    def one_step(ev):
        ev[0].record(stream)
        sv.init_fields(rho_d, u_d, th_d)
        ev[1].record(stream)
        sv.step(NSTEPS)
        ev[2].record(stream)
        sv.moments(mom_d[0], mom_d[1:3], mom_d[3])
        sv.reduce(red_d)
        ev[3].record(stream)

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    warm = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for _ in range(args.warmup):
        flush.zero_()
        one_step(warm)
    torch.cuda.synchronize()

    clocks = ClockSampler(local, args.clocks_out.replace("{rank}", str(rank)) if args.clocks_out else None)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # untimed L2 flush between timed steps
        one_step(evs[k])
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    barrier(world)
    clk = clocks.stop()
    step_ms = [evs[k][0].elapsed_time(evs[k][3]) for k in range(args.steps)]
    loop_ms = [evs[k][1].elapsed_time(evs[k][2]) for k in range(args.steps)]
    total_ms = max_over_ranks(sum(step_ms), world)
    kernel_avg_s = float(np.mean(loop_ms)) / 1e3 / step_launches
    value = world * cells * NSTEPS * args.steps / (total_ms / 1e3) / 1e6

    # sanity: finite and conserved
    red = red_d.cpu().numpy()
    if not np.isfinite(red[:5]).all() or red[5] != 0:
        raise RuntimeError(f"benchmark state not finite: {red}")

    # end-to-end through the C ABI with pinned host buffers
    rho_h = torch.from_numpy(rho).pin_memory()
    u_h = torch.from_numpy(u).pin_memory()
    th_h = torch.from_numpy(th).pin_memory()
    out_h = torch.empty((4, cells), dtype=torch.float64).pin_memory()
    red_h = np.empty(8)
    e2e_times = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        sv.init_fields(rho_h, u_h, th_h)
        sv.step(NSTEPS)
        sv.moments(out_h[0], out_h[1:3], out_h[3])
        sv.reduce(red_h)
        t2 = time.perf_counter()
        if k >= args.warmup:
            e2e_times.append(t2 - t1)
    e2e_total = max_over_ranks(sum(e2e_times), world)
    e2e_value = world * cells * NSTEPS * args.steps / e2e_total / 1e6
    h2d = rho.nbytes + u.nbytes + th.nbytes
    d2h = out_h.numel() * 8 + 6 * 8

    peak, peak_kind = measured_peaks()
    achieved = BYTES_PER_LUP * cells / kernel_avg_s / 1e9
    traffic = profiled_traffic(spl)
    line = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": bench_config(world),
        "wall_s_timed_region": round(wall, 3),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic, "peak_kind": peak_kind,
                     "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                     "bytes_per_update": BYTES_PER_LUP / spl,
                     "update_bound_mlups": round(peak / (BYTES_PER_LUP / spl) * 1e3, 1),
                     "kernel": KERNEL_NAMES.get(spl, "?"),
                     "steps_per_launch": spl,
                     "launches_per_job": {"fused": NSTEPS // spl, "single_step": NSTEPS % spl},
                     "algorithmic_bytes_per_launch": BYTES_PER_LUP * cells,
                     "avg_launch_us": round(kernel_avg_s * 1e6, 3)},
        "e2e": {"value": round(e2e_value, 1), "unit": "MLUPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
    }
    sv.close()
    # rho' of the last timed job (init, 1000 steps, moments: the same bits every job)
    return line, mom_d[0].cpu().numpy()


def cpu_baseline(max_s: float = 90.0):
    """The FP64 oracle as it stands, on all host cores, on the benchmark job itself: init, the
    1000 steps of the 2048^2 grid and rho' (about 22 s on 16 Grace cores).  Returns the timing
    line and the oracle's rho', or None for rho' if the host is so slow that the job would take
    more than max_s seconds (then a bounded number of steps is timed instead)."""
    import oracle
    from paper_1601_08103_gb300 import inputs

    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    rho, u, th = inputs.config_2d(NX, seed=2)
    g0 = oracle.equilibrium(SET, rho, u, th)
    t0 = time.perf_counter()
    g = oracle.step(SET, (NX, NX, 1), TAU, g0, 2)
    probe = (time.perf_counter() - t0) / 2
    full = probe * NSTEPS <= max_s
    n = NSTEPS - 2 if full else int(max(2, min(200, 12.0 / max(probe, 1e-6))))
    t0 = time.perf_counter()
    g = oracle.step(SET, (NX, NX, 1), TAU, g, n)
    dt = time.perf_counter() - t0
    rho_ora = oracle.moments(SET, g)[0] if full else None
    # the same oracle on one thread, a few steps of the same grid (reported beside, not the value)
    oracle.set_threads(1)
    n1 = 4
    t0 = time.perf_counter()
    oracle.step(SET, (NX, NX, 1), TAU, g0, n1)
    dt1 = time.perf_counter() - t0
    what = "the whole job (steps 3..1000 timed)" if full else f"{n} steps"
    line = {"value": round(NX * NX * n / dt / 1e6, 2), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{NX}x{NX} D2Q5 FP64, {what}, {cores} OpenMP threads, {dt:.1f} s",
            "single_thread": {"value": round(NX * NX * n1 / dt1 / 1e6, 2), "unit": "MLUPS",
                              "sample": f"{NX}x{NX} D2Q5 FP64, {n1} steps, 1 thread, {dt1:.1f} s"}}
    return line, rho_ora


def rel_l2_vs_oracle(rho_gpu, rho_ora) -> dict:
    """Relative L2 error of the timed job's rho' (FP32 storage and arithmetic) against the FP64
    oracle run of the same job (the space L2 norm of Sec. 9 at the final time)."""
    if rho_ora is None:
        return {"value": None, "reason": "oracle job too slow on this host; not compared"}
    err = float(np.linalg.norm(rho_gpu - rho_ora) / np.linalg.norm(rho_ora))
    return {"value": err, "field": "rho'", "against": "FP64 oracle, the same 1000-step job", "tolerance": 1e-5}


def forms_3d():
    """Mixed-precision storage forms on the 3D configuration (D3Q7, 384^3, tau = 0.55, Gaussian
    pulse amplitude 1e-3 width 16, 500 steps): MLUPS of each storage and relative L2 of rho'
    against the FP64 run on the same GPU (FP64 itself is held to the oracle by the tests)."""
    import torch

    import paper_1601_08103_gb300 as lee
    from paper_1601_08103_gb300 import inputs

    n, steps = 384, 500
    cells = n ** 3
    rho, u, th = inputs.config_3d(n, seed=3)
    dev = torch.device("cuda")
    rho_d, u_d, th_d = (torch.from_numpy(a).to(dev) for a in (rho, u, th))
    out = {}
    ref = None
    stream = torch.cuda.current_stream()
    # (label, storage, environment at create time): the default kernels, and the TMA-fed two-step
    # tile that LEE_T3_TMA=1 selects (measured slower; reported for the record)
    forms = [(st, st, {}) for st in ("f64", "f32", "f16", "bf16", "bfp16")]
    forms += [("f32_tma_tile", "f32", {"LEE_T3_TMA": "1"}), ("bfp16_tma_tile", "bfp16", {"LEE_T3_TMA": "1"})]
    for label, storage, env in forms:
        saved = {k: os.environ.get(k) for k in env}
        os.environ.update(env)
        try:
            sv = lee.Solver("D3Q7", (n, n, n), 0.55, storage=storage, stream=stream)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        with sv:
            sv.init_fields(rho_d, u_d, th_d)
            sv.step(2)
            sv.init_fields(rho_d, u_d, th_d)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            sv.step(steps)
            e1.record(stream)
            r = torch.empty(cells, dtype=torch.float64, device=dev)
            sv.moments(r, None, None)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            spl = sv.steps_per_launch
        if label == "f64":
            ref = r
        err = float(torch.linalg.norm(r - ref) / torch.linalg.norm(ref))
        bpl = 2 * 7 * lee.STORAGE_BYTES[storage]
        out[label] = {"mlups": round(cells * steps / (ms / 1e3) / 1e6, 1),
                        "gbs": round(bpl * cells * steps / (ms / 1e3) / 1e9, 1), "rel_l2_rho_vs_f64": err,
                        "steps_per_launch": spl, "bytes_per_update": round(bpl / max(spl, 1), 3)}
    for label in ("f16", "bf16", "bfp16", "f32_tma_tile", "bfp16_tma_tile"):
        out[label]["mlups_gain_vs_f32"] = round(out[label]["mlups"] / out["f32"]["mlups"], 3)
    return {"workload": "3D D3Q7 periodic 384^3, tau=0.55, pulse A=1e-3 w=16, 500 steps", "storage": out,
            "error_reference": "the FP64 run on the GPU, which the tests hold to the oracle within 1e-12 "
                               "(test_full_size_3d_config_against_oracle also checks every storage against "
                               "the oracle directly)"}


def _device_config_2d(n: int, seed: int = 2):
    """The 2D configuration's field (Gaussian pulse A = 1e-3, w = 32, plus 8 density plane waves of
    amplitude 1e-4, wavelength 16-256 cells) on an n x n grid, drawn from the same random sequence
    as inputs.config_2d but evaluated on the device (8192^2 would need gigabytes on the host)."""
    import torch

    rng = np.random.default_rng(seed)
    c = rng.uniform(0, n, size=2)
    rho = _device_pulse((n, n, 1), 1e-3, 32.0, [c[0], c[1], 0.0])
    lo, hi = max(1.0, n / 256.0), max(1.0, n / 16.0)
    ax = torch.arange(n, dtype=torch.float64, device="cuda")
    for _ in range(8):
        while True:
            kmag = rng.uniform(lo, hi)
            ang = rng.uniform(0, 2 * np.pi)
            m = (int(round(kmag * np.cos(ang))), int(round(kmag * np.sin(ang))))
            if m[0] != 0 or m[1] != 0:
                break
        ph = rng.uniform(0, 2 * np.pi)
        arg = (2 * np.pi * m[0] / n) * ax[None, :] + (2 * np.pi * m[1] / n) * ax[:, None] + ph
        rho += 1e-4 * torch.cos(arg).reshape(-1)
    return rho


def forms_mixed_2d(n: int = 8192, steps: int = 1000):
    """The mixed-precision storage forms on a 2D grid far beyond L2 (D2Q5, n^2, tau = 0.6, the 2D
    configuration's pulse and plane waves, 1000 steps): MLUPS, bytes per update of the kernel that
    ran, and the relative L2 error of rho' against the FP64 run."""
    import torch

    import paper_1601_08103_gb300 as lee

    cells = n * n
    stream = torch.cuda.current_stream()
    rho = _device_config_2d(n)
    u = torch.zeros((2, cells), dtype=torch.float64, device="cuda")
    th = torch.zeros(cells, dtype=torch.float64, device="cuda")
    out, ref = {}, None
    for storage in ("f64", "f32", "f16", "bfp16"):
        with lee.Solver("D2Q5", (n, n, 1), 0.6, storage=storage, stream=stream) as sv:
            sv.init_fields(rho, u, th)
            sv.step(8)
            sv.init_fields(rho, u, th)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            sv.step(steps)
            e1.record(stream)
            r = torch.empty(cells, dtype=torch.float64, device="cuda")
            sv.moments(r, None, None)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            spl = sv.steps_per_launch
        if ref is None:
            ref = r
        bpl = 2 * 5 * lee.STORAGE_BYTES[storage]
        out[storage] = {"mlups": round(cells * steps / (ms / 1e3) / 1e6, 1), "steps_per_launch": spl,
                        "bytes_per_update": round(bpl / spl, 3),
                        "gbs_algorithmic_per_launch": round(bpl * cells * steps / spl / (ms / 1e3) / 1e9, 1),
                        "rel_l2_rho_vs_f64": float(torch.linalg.norm(r - ref) / torch.linalg.norm(ref))}
        del r
        torch.cuda.empty_cache()
    for storage in ("f16", "bfp16"):
        out[storage]["mlups_gain_vs_f32"] = round(out[storage]["mlups"] / out["f32"]["mlups"], 3)
    return {"workload": f"2D D2Q5 periodic {n}x{n}, tau=0.6, pulse+8 plane waves, {steps} steps", "storage": out,
            "error_reference": "the FP64 run on the GPU (held to the oracle by the tests)"}


def _device_pulse(shape, amplitude: float, width: float, center):
    """amplitude * exp(-|x - center|^2 / width^2) with periodic minimum-image distances, built on
    the device (the large grids below would need gigabytes of host coordinates)."""
    import torch

    dims = (list(shape) + [1, 1])[:3]
    r2 = torch.zeros((dims[2], dims[1], dims[0]), dtype=torch.float64, device="cuda")
    for a in range(3):
        if dims[a] == 1:
            continue
        ax = torch.arange(dims[a], dtype=torch.float64, device="cuda")
        d = torch.remainder(ax - center[a] + dims[a] / 2.0, dims[a]) - dims[a] / 2.0
        view = [1, 1, 1]
        view[2 - a] = dims[a]
        r2 = r2 + (d * d).view(view)
    return (amplitude * torch.exp(-r2 / (width * width))).reshape(-1)


def forms_configs():
    """The other configurations of the workload table, each timed alone with CUDA events (inputs
    resident, after a short warm-up): 1D D1Q3 N = 1024 FP64 (on-chip, time per step) and
    N = 2^28 FP64 (the 1D roofline run), 2D D2Q5 2048^2 FP64, 2D D2Q5 8192^2 FP32 (working set
    2.7 GB, far beyond L2) and 3D D3Q19 256^3 FP32 (the largest velocity set)."""
    import torch

    import paper_1601_08103_gb300 as lee

    runs = [("1d_d1q3_f64_1024", "D1Q3", (1024, 1, 1), "f64", 0.8, 2000, 16.0),
            ("1d_d1q3_f64_2^28", "D1Q3", (1 << 28, 1, 1), "f64", 0.8, 20, 20.0),
            ("2d_d2q5_f64_2048", "D2Q5", (2048, 2048, 1), "f64", 0.6, 1000, 32.0),
            ("2d_d2q5_f32_8192", "D2Q5", (8192, 8192, 1), "f32", 0.6, 1000, 32.0),
            ("3d_d3q19_f32_256", "D3Q19", (256, 256, 256), "f32", 0.55, 100, 16.0)]
    out = {}
    stream = torch.cuda.current_stream()
    for key, name, shape, storage, tau, steps, w in runs:
        info = lee.lee_velset_info(name)
        cells = int(np.prod(shape))
        rho = _device_pulse(shape, 1e-3, w, [n / 2.7 for n in shape])
        u = torch.zeros((info["D"], cells), dtype=torch.float64, device="cuda")
        th = torch.zeros(cells, dtype=torch.float64, device="cuda")
        with lee.Solver(name, shape, tau, storage=storage, stream=stream) as sv:
            sv.init_fields(rho, u, th)
            sv.step(4)
            sv.init_fields(rho, u, th)
            del rho, u, th
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            sv.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            finite = sv.check_finite()
            spl = sv.steps_per_launch
        bpl = 2 * info["q"] * lee.STORAGE_BYTES[storage]
        out[key] = {"cells": cells, "steps": steps, "ms": round(ms, 3), "us_per_step": round(ms * 1e3 / steps, 3),
                    "mlups": round(cells * steps / (ms / 1e3) / 1e6, 1),
                    "gbs": round(bpl * cells * steps / (ms / 1e3) / 1e9, 1), "bytes_per_lup": bpl,
                    "steps_per_launch": spl, "finite": bool(finite)}
        torch.cuda.empty_cache()
    # the measured FP64 fma rate: the roofline of the FP64 storage forms, whose collision is FP64
    out["fp64_fma_peak"] = {"tflops": round(lee.lee_probe_fp64_fma(1 << 16) / 1e12, 4),
                            "how": "8 independent FP64 fma chains per thread, 8 x 256 threads per SM, CUDA events"}
    return out


def forms_stability():
    """The von Neumann scan of Theorem 1 (Sec. 7) on the GPU: grid points per second and the
    extreme values of the spectral radius and kappa_W, for tau = 1/2 and 0.7."""
    import torch

    import paper_1601_08103_gb300 as lee

    out = {}
    for name, m in (("D2Q5", 512), ("D3Q7_DI", 48), ("D3Q19", 48)):
        info = lee.lee_velset_info(name)
        n = m ** info["D"]
        rho = torch.empty(n, dtype=torch.float64, device="cuda")
        kap = torch.empty(n, dtype=torch.float64, device="cuda")
        nu = torch.empty(n, dtype=torch.float64, device="cuda")
        for tau in (0.5, 0.7):
            lee.lee_stability_scan(name, tau, m, rho, None, kap, nu)  # warm-up (local memory set-up)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lee.lee_stability_scan(name, tau, m, rho, None, kap, nu)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            out[f"{name}_m{m}_tau{tau}"] = {"points": n, "s": round(dt, 4), "points_per_s": round(n / dt, 1),
                                            "rho_max": float(rho.max()), "kappa_max": float(kap.max()),
                                            "nu_max": float(nu.max())}
    return out


def forms_split():
    """Split storage on the velocity set it is for: D3Q19 256^3, tau = 0.55, Gaussian pulse
    (A = 1e-3, w = 16), 200 steps, in FP32, FP16 and split16 (FP32 moments + FP16 non-equilibrium
    parts): MLUPS, algorithmic GB/s, bytes per cell and copy, and the relative L2 error of rho'
    against the FP64 run on the same GPU."""
    import torch

    import paper_1601_08103_gb300 as lee

    name, n, steps = "D3Q19", 256, 200
    info = lee.lee_velset_info(name)
    cells = n ** 3
    stream = torch.cuda.current_stream()
    rho = _device_pulse((n, n, n), 1e-3, 16.0, [n / 2.7] * 3)
    u = torch.zeros((3, cells), dtype=torch.float64, device="cuda")
    th = torch.zeros(cells, dtype=torch.float64, device="cuda")
    out, ref = {}, None
    for storage in ("f64", "f32", "f16", "split16", "bfp16"):
        with lee.Solver(name, (n, n, n), 0.55, storage=storage, stream=stream) as sv:
            sv.init_fields(rho, u, th)
            sv.step(2)
            sv.init_fields(rho, u, th)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            sv.step(steps)
            e1.record(stream)
            r = torch.empty(cells, dtype=torch.float64, device="cuda")
            sv.moments(r, None, None)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
        if ref is None:
            ref = r
        bpc = lee.state_bytes_per_cell(3, info["q"], storage)
        out[storage] = {"mlups": round(cells * steps / (ms / 1e3) / 1e6, 1),
                        "gbs": round(2 * bpc * cells * steps / (ms / 1e3) / 1e9, 1), "bytes_per_cell_copy": bpc,
                        "rel_l2_rho_vs_f64": float(torch.linalg.norm(r - ref) / torch.linalg.norm(ref))}
    return {"workload": "3D D3Q19 periodic 256^3, tau=0.55, pulse A=1e-3 w=16, 200 steps", "storage": out}


def forms_slab(n: int = 384, steps: int = 100):
    """Slab decomposition of the 3D configuration's grid (D3Q7 n^3, FP32, tau = 0.55) on one GPU:
    the domain cut along z into 1, 2 and 4 slabs held in this process, advanced by
    lee_lbm_slab_step (per step: pack the crossing populations, copy each message into the
    receiving slab's own buffer, unpack, one one-step launch per slab), against the single-domain
    one-step run of the same grid (LEE_TB_STEPS=1); results equal bit for bit."""
    import torch

    import paper_1601_08103_gb300 as lee
    from paper_1601_08103_gb300 import slab

    stream = torch.cuda.current_stream()
    cells = n ** 3
    rho = _device_pulse((n, n, n), 1e-3, 16.0, [n / 2.7] * 3)
    u = torch.zeros((3, cells), dtype=torch.float64, device="cuda")
    th = torch.zeros(cells, dtype=torch.float64, device="cuda")
    out = {}

    def timed(run):
        run()  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        run()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    old = os.environ.get("LEE_TB_STEPS")
    os.environ["LEE_TB_STEPS"] = "1"
    try:
        with lee.Solver("D3Q7", (n, n, n), 0.55, storage="f32", stream=stream) as sv:
            sv.init_fields(rho, u, th)
            ms = timed(lambda: sv.step(steps))
            ref = torch.empty(cells, dtype=torch.float64, device="cuda")
            sv.init_fields(rho, u, th)
            sv.step(steps)
            sv.moments(ref, None, None)
    finally:
        if old is None:
            del os.environ["LEE_TB_STEPS"]
        else:
            os.environ["LEE_TB_STEPS"] = old
    out["single_domain_one_step"] = {"mlups": round(cells * steps / (ms / 1e3) / 1e6, 1), "ms": round(ms, 3)}
    for count in (1, 2, 4):
        parts = slab.partition(n, count)
        slabs = [lee.Solver("D3Q7", (n, n, c), 0.55, storage="f32", bc="slab", stream=stream) for _, c in parts]
        try:
            def init():
                for sv, (z0, c) in zip(slabs, parts):
                    sl = slice(z0 * n * n, (z0 + c) * n * n)
                    sv.init_fields(rho[sl].contiguous(), u[:, sl].contiguous(), th[sl].contiguous())
            init()
            ms = timed(lambda: lee.lee_lbm_slab_step(slabs, steps))
            init()
            lee.lee_lbm_slab_step(slabs, steps)
            got = torch.empty(cells, dtype=torch.float64, device="cuda")
            for sv, (z0, c) in zip(slabs, parts):
                sv.moments(got[z0 * n * n:(z0 + c) * n * n], None, None)
            torch.cuda.synchronize()
            crossing, plane, nbytes = slabs[0].slab_info()
        finally:
            for sv in slabs:
                sv.close()
        out[f"slabs_{count}"] = {"mlups": round(cells * steps / (ms / 1e3) / 1e6, 1), "ms": round(ms, 3),
                                 "halo_bytes_per_step": 2 * count * nbytes,
                                 "bit_equal_to_single_domain": bool(torch.equal(got, ref))}
    return {"workload": f"3D D3Q7 periodic {n}^3 FP32 cut along z, {steps} steps, one GPU (in-process slabs)",
            "slabs": out}


def forms_batched(steps: int = 1000):
    """Batched 2D form: 96 periodic D2Q5 domains (sizes from {128, ..., 1024}^2, tau in
    [0.52, 1.2], one pulse each, seed 4), FP32, `steps` steps, in one batched launch per step
    replayed from one CUDA graph, against one batched launch per step without a graph and against
    96 sequential plain launches per step; error of rho' against the FP64 batch."""
    import torch

    import paper_1601_08103_gb300 as lee
    from paper_1601_08103_gb300 import inputs

    specs = inputs.batched_2d_specs(96, seed=4)
    doms = [(s["nx"], s["ny"], s["tau"]) for s in specs]
    fields = [tuple(torch.from_numpy(a).cuda() for a in inputs.batched_2d_fields(s)) for s in specs]
    stream = torch.cuda.current_stream()
    out = {}
    rho_by = {}
    out_shape = None
    for storage, mode in (("f64", "graph"), ("f32", "sequential"), ("f32", "launch"), ("f32", "graph")):
        with lee.Batch("D2Q5", storage, doms, stream=stream) as b:
            cells = b.cells
            for d, f in enumerate(fields):
                b.init_fields(d, *f)
            b.step(steps, mode)  # warm-up run: tuning, graph capture
            for d, f in enumerate(fields):
                b.init_fields(d, *f)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            b.step(steps, mode)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            rho = torch.cat([torch.empty(nx * ny, dtype=torch.float64, device="cuda") for nx, ny, _ in doms])
            off = 0
            for d, (nx, ny, _) in enumerate(doms):
                b.moments(d, rho[off: off + nx * ny], None, None)
                off += nx * ny
            torch.cuda.synchronize()
            shape = b.tune() if mode != "sequential" else None
            if mode == "graph" and storage == "f32":
                out_shape = b.tune_shape()
        key = f"{storage}_{mode}"
        out[key] = {"mlups": round(cells * steps / (ms / 1e3) / 1e6, 1), "ms": round(ms, 3),
                    "gbs": round(2 * 5 * lee.STORAGE_BYTES[storage] * cells * steps / (ms / 1e3) / 1e9, 1)}
        if shape:
            out[key]["tuned_threads_cells_per_thread"] = list(shape)
        rho_by[(storage, mode)] = rho
    # the fair baseline: every domain through its own best single-domain path (lee_lbm_step, four
    # fused steps per launch replayed from a CUDA graph), one domain after the other
    solvers = [lee.Solver("D2Q5", (nx, ny, 1), tau, storage="f32", stream=stream) for nx, ny, tau in doms]
    for sv, f in zip(solvers, fields):
        sv.init_fields(*f)
        sv.step(steps)  # warm-up: graph capture
        sv.init_fields(*f)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for sv in solvers:
        sv.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_pd = e0.elapsed_time(e1)
    rho_pd = torch.cat([torch.empty(nx * ny, dtype=torch.float64, device="cuda") for nx, ny, _ in doms])
    off = 0
    for sv, (nx, ny, _) in zip(solvers, doms):
        sv.moments(rho_pd[off: off + nx * ny], None, None)
        off += nx * ny
        sv.close()
    torch.cuda.synchronize()
    out["f32_per_domain_best"] = {"mlups": round(cells * steps / (ms_pd / 1e3) / 1e6, 1), "ms": round(ms_pd, 3),
                                  "bit_equal_to_batched": bool(torch.equal(rho_pd, rho_by[("f32", "graph")]))}
    ref = rho_by[("f64", "graph")]
    for (storage, mode), r in rho_by.items():
        out[f"{storage}_{mode}"]["rel_l2_rho_vs_f64"] = float(torch.linalg.norm(r - ref) / torch.linalg.norm(ref))
    seq = out["f32_sequential"]["ms"]
    return {"workload": f"96 periodic D2Q5 domains, {cells} cells, FP32, {steps} steps", "modes": out,
            "tuned_shape": out_shape,
            "speedup_graph_vs_sequential": round(seq / out["f32_graph"]["ms"], 3),
            "speedup_launch_vs_sequential": round(seq / out["f32_launch"]["ms"], 3),
            "speedup_graph_vs_per_domain_best": round(ms_pd / out["f32_graph"]["ms"], 3)}


def forms_learned(n: int = 1024, steps: int = 3000):
    """Learned-boundary form: the 1024^2 open D2Q5 grid (FP32, tau 0.6, seeded off-centre pulses,
    3000 steps) with the zero-incoming edge, a 24-cell sponge frame (1072^2 grid) and the trained
    boundary network shipped in paper_1601_08103_gb300/data, against the light-cone-enlarged FP64
    periodic run: relative space-time L2 error of rho' and MLUPS per physical cell."""
    import paper_1601_08103_gb300 as lee
    from paper_1601_08103_gb300 import learned_boundary

    params = np.load(os.path.join(ROOT, "paper_1601_08103_gb300", "data", "boundary_d2q5_tau0.6.npy"))
    return learned_boundary.evaluate(lee, params.astype(np.float32), n=n, steps=steps)


CASES = {
    # name: (set, shape, storage, tau)
    "d1q3_f64": ("D1Q3", (1024, 1, 1), "f64", 0.8),
    "d2q5_f32": ("D2Q5", (2048, 2048, 1), "f32", 0.6),
    "d2q5_f64": ("D2Q5", (2048, 2048, 1), "f64", 0.6),
    "d3q7_f32": ("D3Q7", (384, 384, 384), "f32", 0.55),
    "d3q7_f32_256": ("D3Q7", (256, 256, 256), "f32", 0.55),
    "d3q7_f64": ("D3Q7", (384, 384, 384), "f64", 0.55),
    "d3q7_f16": ("D3Q7", (384, 384, 384), "f16", 0.55),
    "d3q7_bf16": ("D3Q7", (384, 384, 384), "bf16", 0.55),
    "d3q19_f32": ("D3Q19", (256, 256, 256), "f32", 0.55),
    "d3q19_f16": ("D3Q19", (256, 256, 256), "f16", 0.55),
    "d3q19_split16": ("D3Q19", (256, 256, 256), "split16", 0.55),
    "d3q13_f32": ("D3Q13", (256, 256, 256), "f32", 0.55),
    "d3q13_split16": ("D3Q13", (256, 256, 256), "split16", 0.55),
    "d2q5_f32_4096": ("D2Q5", (4096, 4096, 1), "f32", 0.6),
    "d2q5_f32_8192": ("D2Q5", (8192, 8192, 1), "f32", 0.6),
    "d2q5_f16_8192": ("D2Q5", (8192, 8192, 1), "f16", 0.6),
    "d2q5_f16_4096": ("D2Q5", (4096, 4096, 1), "f16", 0.6),
    "d2q5_bfp16_8192": ("D2Q5", (8192, 8192, 1), "bfp16", 0.6),
    "d2q5_bfp16": ("D2Q5", (2048, 2048, 1), "bfp16", 0.6),
    "d2q5_bfp16_4096": ("D2Q5", (4096, 4096, 1), "bfp16", 0.6),
    "d3q7_bfp16": ("D3Q7", (384, 384, 384), "bfp16", 0.55),
    "d3q7_bfp16_256": ("D3Q7", (256, 256, 256), "bfp16", 0.55),
    "d3q19_bfp16": ("D3Q19", (256, 256, 256), "bfp16", 0.55),
    "d3q7_f32_odd": ("D3Q7", (385, 383, 381), "f32", 0.55),
    "d2q5_learned_1024": ("D2Q5", (1024, 1024, 1), "f32", 0.6, "open_learned"),
    "d2q5_zero_1024": ("D2Q5", (1024, 1024, 1), "f32", 0.6, "open_zero"),
}


def run_case(args):
    """One configuration alone (for profiling): warmup LBM steps, then --steps LBM steps timed
    with CUDA events; prints a small JSON line (not a benchmark line)."""
    import torch

    import paper_1601_08103_gb300 as lee
    from paper_1601_08103_gb300 import inputs

    name, shape, storage, tau = CASES[args.case][:4]
    bc = CASES[args.case][4] if len(CASES[args.case]) > 4 else "periodic"
    lee.load()
    stream = torch.cuda.current_stream()
    D = lee.lee_velset_info(name)["D"]
    cells = int(np.prod(shape))
    c = [n / 2.7 for n in shape]
    rho = inputs.gaussian_pulse(shape, 1e-3, 16.0, c)
    u, th = inputs.zero_rest(D, cells)
    with lee.Solver(name, shape, tau, storage=storage, bc=bc, stream=stream) as sv:
        if bc == "open_learned":
            from paper_1601_08103_gb300 import learned_boundary

            sv.set_boundary_mlp(learned_boundary.he_init(0))
        sv.init_fields(rho, u, th)
        sv.step(args.warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sv.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ok = sv.check_finite()
    q = lee.lee_velset_info(name)["q"]
    bpl = 2 * lee.state_bytes_per_cell(D, q, storage)
    print(json.dumps({"case": args.case, "cells": cells, "steps": args.steps, "ms": ms, "finite": ok,
                      "mlups": cells * args.steps / (ms / 1e3) / 1e6,
                      "gbs": bpl * cells * args.steps / (ms / 1e3) / 1e9}), flush=True)
    return 0 if ok else 1


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle as it stands on the host cores (rank 0 only)."""
    if rank != 0:
        return None
    import oracle
    from paper_1601_08103_gb300 import inputs

    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    rho, u, th = inputs.config_2d(NX, seed=2)
    g0 = oracle.equilibrium(SET, rho, u, th)
    sample_steps = 3
    for _ in range(args.warmup):
        oracle.step(SET, (NX, NX, 1), TAU, g0, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.step(SET, (NX, NX, 1), TAU, g0, sample_steps)
    dt = time.perf_counter() - t0
    value = NX * NX * sample_steps * args.steps / dt / 1e6
    sample = (f"{NX}x{NX} D2Q5 FP64, {sample_steps} steps per timed step, {cores} OpenMP threads "
              "(oracle: plain FP64 C restatement of the paper's update, bounded sample)")
    return {"impl": "reference", "metric": METRIC,
            "value": round(value, 2), "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(world),
            "cpu_baseline": {"value": round(value, 2), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 2), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", choices=sorted(CASES), help="time one configuration alone (profiling)")
    ap.add_argument("--clocks-out", default=None,
                    help="keep the nvidia-smi clock samples of the timed region in this CSV ({rank} = rank)")
    args = ap.parse_args(argv)
    if args.case:
        return run_case(args)
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return 0
    line, rho_gpu = run_ours(args, rank, world, local)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"], rho_ora = cpu_baseline()
            line["rel_l2_vs_f64"] = rel_l2_vs_oracle(rho_gpu, rho_ora)
        if world == 1 and not args.no_forms:
            line["forms"] = forms_3d()
            line["forms_mixed_2d"] = forms_mixed_2d()
            line["forms_configs"] = forms_configs()
            line["forms_stability"] = forms_stability()
            line["forms_split"] = forms_split()
            line["forms_batched"] = forms_batched()
            line["forms_slab"] = forms_slab()
            line["forms_learned"] = forms_learned()
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
