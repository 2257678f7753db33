#!/usr/bin/env python
"""Benchmark of the JAGP VMC hot path on one GB300 (or N, one process each).

A step is one pass of the whole path over every walker: one Metropolis sweep
(every electron proposed once: orbital evaluation, proposed rows/columns of
G~, sequential Sherman-Morrison acceptance, lambda products of the accepted
rows), the FP64 refresh of G~^{-1}, log|det| and J, the local energy of every
walker and the per-sweep reductions.

Workload (N=1): the plain-FP64 VMC configuration with 16 He atoms in a 10 bohr
cube, N = 32 electrons (16 up, 16 down), 20 s/p/d Gaussians per atom (L = 320),
dense random symmetric lambda, one- and two-body Jastrow, 4096 walkers.
The walker state (~1 GB) is larger than L2, so no flush is needed between
steps.  Under torchrun each rank runs its own 4096 walkers (weak scaling, no
data-path collective; a barrier and a max-reduction of the timings only).

Prints one JSON line (rank 0).  Each timed region is an NVTX push/pop range
(fp64, mixed, fp64tc, batched, forces, large, large_forces), so that a profiler
can keep to it (ncu --nvtx --nvtx-include "batched/").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "walker-electron moves/s and E_L+forces/s, mixed/batched vs plain FP64 on 1 GB300"
UNIT = "walker-electron moves/s"
WORKLOAD = ("plain FP64 VMC: 16 He atoms in a 10 bohr cube (min separation 1.5), N=32 (16 up, 16 down), "
            "20 s/p/d Gaussians/atom (L=320), dense random symmetric lambda, J1 + J2, 4096 walkers/GPU")
# FP64 CUDA-core peak of one GB300 (no measured value available): 1.25 TFLOP/s nominal
FP64_PEAK_TFLOPS = 1.25


def _bf16_sustained_peak():
    """BF16 dense tensor-core peak for kernels timed inside a long step: the
    sustained cuBLAS figure of MEASURED_PEAKS.json when that file is present,
    else the fallback 1.7 PFLOP/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            v = float(json.load(fh)["bf16_tflops_sustained"])
        if v > 0:
            return v, "measured BF16 sustained (MEASURED_PEAKS.json bf16_tflops_sustained)"
    except (OSError, KeyError, ValueError, TypeError):
        pass
    return 1700.0, "fallback BF16 sustained (no MEASURED_PEAKS file)"


BF16_SUSTAINED_TFLOPS, BF16_PEAK_SOURCE = _bf16_sustained_peak()
# BF16 slice-pair products per element of the mixed path's lambda products: the
# up-spin rows (phi^T lambda, FP32 result) take 10, the down-spin rows (lambda
# phi, two-float result) 15; accepted moves are split between the spins in
# proportion to their electron counts when the issued work is counted
PAIRS_UP, PAIRS_DN = 10, 15
NO_AUTOTUNE = False  # --no-autotune: time the shape heuristics' tiles


def fixed_pairs(sysm):
    return (PAIRS_UP * sysm.n_up + PAIRS_DN * sysm.n_dn) / sysm.N
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "k_lambda_rows_C2_traffic.txt")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def emit(obj):
    print(json.dumps(obj), flush=True)


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # raw samples go to $JAGP_CLOCK_LOG_DIR (default: the temporary directory)
        log_dir = os.environ.get("JAGP_CLOCK_LOG_DIR") or tempfile.gettempdir()
        self.path = os.path.join(log_dir, f"jagp_clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                p = [t.strip() for t in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for name, v in zip(names, p[5:9]):
                    if v.lower() in ("active", "0x1") or v == "1":
                        reasons.add(name)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU oracle (test infrastructure) timed on the host cores
# ----------------------------------------------------------------------------
def oracle_rate(sysm, target_s: float = 15.0, max_walkers: int = 4096):
    """Oracle VMC sweeps + local energies on a bounded sample of the same
    workload (up to all of its walkers, then more sweeps) sized to roughly
    target_s seconds; returns (moves/s, e_L/s, cores, sample description, seconds)."""
    import oracle
    import synth
    o = oracle.Oracle(sysm)
    cores = oracle.max_threads()
    Ws, sweeps = max(cores, 8), 1
    while True:
        x = synth.init_walkers(sysm, Ws, seed=0)
        t0 = time.perf_counter()
        o.vmc(x, sweeps, seed=0, sweep0=0, walker0=0, record_eL=True, nthreads=cores)
        dt = time.perf_counter() - t0
        if dt >= target_s * 0.5:
            break
        grow = min(8.0, max(2.0, target_s / max(dt, 1e-3)))
        if Ws < max_walkers:
            Ws = min(max_walkers, int(Ws * grow))
        else:
            sweeps = int(sweeps * grow) + 1
    moves = Ws * sweeps * sysm.N
    return (moves / dt, Ws * sweeps / dt, cores,
            f"{Ws} walkers x {sweeps} sweep(s) (+ e_L per walker and sweep) of the same system", dt)


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return os.uname().machine


# ----------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands
# ----------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import synth
    sysm = synth.config2()
    import oracle
    o = oracle.Oracle(sysm)
    cores = oracle.max_threads()
    # size one step so that the whole --steps/--warmup run stays near two minutes
    per_step = max(1.0, 120.0 / (args.steps + args.warmup))
    Ws = max(cores, 8)
    x = synth.init_walkers(sysm, Ws, seed=0)
    t0 = time.perf_counter()
    o.vmc(x, 1, seed=0, record_eL=True, nthreads=cores)
    dt = time.perf_counter() - t0
    Ws = int(min(4096, max(Ws, Ws * per_step / max(dt, 1e-3))))
    x = synth.init_walkers(sysm, Ws, seed=0)
    for k in range(args.warmup):
        o.vmc(x, 1, seed=0, sweep0=k, record_eL=True, nthreads=cores)
    t0 = time.perf_counter()
    for k in range(args.steps):
        o.vmc(x, 1, seed=0, sweep0=args.warmup + k, record_eL=True, nthreads=cores)
    dt = time.perf_counter() - t0
    value = Ws * sysm.N * args.steps / dt
    sample = f"{Ws} walkers per step (of 4096), 1 sweep + e_L per walker, {cores} threads, {cpu_model()}"
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
          "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
          "config": {"workload": WORKLOAD, "sample_walkers": Ws},
          "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})
    return 0


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("k_lambda.cu",):
        h.update(open(os.path.join(ROOT, "paper_2002_07401_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(src_hash):
    try:
        d = json.load(open(PROFILE_TRAFFIC))
    except (OSError, ValueError):
        return None, None
    if d.get("source_hash") != src_hash:
        return None, None
    return d.get("dram_bytes_per_accepted_row"), d


def timed_sweeps(pg, torch, dist, sysm, W, walker0, x0, prec, steps, warmup, ws, dev, local, profile_kernel,
                 fp64_tc=False, label=None, pin=None):
    """Warm up, then time `steps` sweeps (+ local energies) with CUDA events on the
    launching stream; the profiled kernel class is bracketed by event pairs.  The
    timed sweeps form the NVTX range `label` (default: fp64, mixed or fp64tc).
    `pin` (a tuning dict) replaces the autotuner's choices."""
    if label is None:
        label = "fp64tc" if fp64_tc else ("mixed" if prec == pg.JAGP_PREC_MIXED else "fp64")
    g = pg.JAGP(sysm, W, seed=0, precision=prec, fp64_tc=fp64_tc)
    h = g.h
    if pin is not None:
        g.set_tuning(pin)
        tuning = dict(pin, pinned=True)
    else:
        tuning = None if NO_AUTOTUNE else g.autotune()  # tile choices for this system and walker count
    r = g.positions(x0)
    stream = torch.cuda.current_stream()
    eL = torch.empty((1, W), dtype=torch.float64, device=dev)
    acc_steps = torch.empty((steps, 4), dtype=torch.float64, device=dev)
    acc_tmp = torch.empty((1, 4), dtype=torch.float64, device=dev)
    pg.jagp_eval(h, r, W, g.state)
    for k in range(warmup):
        pg.vmc_sweep(h, r, g.state, W, 1, walker0, k, eL, acc_tmp)
    torch.cuda.synchronize()
    bits = g.status()
    pg.jagp_profile(h, profile_kernel, True)
    pg.jagp_profile_read(h)  # clear
    n0 = pg.jagp_launch_count(h)
    e_start, e_stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push(label)
        e_start.record(stream)
        for k in range(steps):
            pg.vmc_sweep(h, r, g.state, W, 1, walker0, warmup + k, eL, acc_steps[k:k + 1])
        e_stop.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
    launches = pg.jagp_launch_count(h) - n0
    prof_ms, prof_n = pg.jagp_profile_read(h)
    pg.jagp_profile(h, profile_kernel, False)
    ms = e_start.elapsed_time(e_stop)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    acc = acc_steps.cpu().numpy()
    bits |= g.status()
    return {"g": g, "r": r, "eL": eL, "ms": ms, "ms_max": float(t.item()), "launches": launches,
            "prof_ms": prof_ms, "prof_n": prof_n, "accepted": float(acc[:, 2].sum()), "bits": bits,
            "clocks": clk.summary(), "tuning": tuning}


FORCES_WORKLOAD = ("adjoint gradients: 64 He atoms in a 16 bohr cube, N=128 (64 up, 64 down), 24 s/p/d Gaussians/"
                   "atom (L=1536), 2048 walkers/GPU; per configuration e_L, the ionic force vector (Hellmann-Feynman "
                   "+ Pulay, Eq. forces:aad without space warp), d log|Psi|/d lambda and d log|Psi|/d b")


def forces_bench(pg, torch, dist, args, dev, rank, ws, local, fp64_tc=False):
    """E_L + forces per second: one step = jagp_grad over all walkers with the
    force-estimator seeds (sE = 1/M, sL = 2 (e_L - <e_L>)/M from the walkers'
    local energies), producing e_L, dE/dR, d log|Psi|/d lambda and d/d b."""
    import numpy as np
    import synth
    sysm = synth.config4()
    W = args.force_walkers
    x0 = np.ascontiguousarray(synth.init_walkers(sysm, W * ws, seed=0)[rank * W:(rank + 1) * W])
    g = pg.JAGP(sysm, W, seed=0, fp64_tc=fp64_tc)
    r = g.positions(x0)
    g.eval(r)
    eL, _ = g.sweep(r, 1, walker0=rank * W, sweep0=0)
    e = eL[0]
    sE = torch.full((W,), 1.0 / W, dtype=torch.float64, device=dev)
    sL = 2.0 * (e - e.mean()) / W
    work = torch.empty(pg.jagp_grad_workspace_bytes(g.h, W), dtype=torch.uint8, device=dev)
    f64 = dict(dtype=torch.float64, device=dev)
    L, na = sysm.L, sysm.n_atoms
    out = dict(eL=torch.empty(W, **f64), lam=torch.empty((L, L), **f64), jas=torch.empty(3, **f64),
               R=torch.empty((na, 3), **f64))
    call = lambda: pg.jagp_grad(g.h, r, g.state, W, work, sL, sE, out["eL"], out["lam"], out["jas"], out["R"])  # noqa
    for _ in range(args.force_warmup):
        call()
    torch.cuda.synchronize()
    pg.jagp_profile(g.h, pg.KERNEL_LAMBDA_ROWS, True)
    pg.jagp_profile_read(g.h)
    n0 = pg.jagp_launch_count(g.h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("forces")
    e0.record()
    for _ in range(args.force_steps):
        call()
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches = pg.jagp_launch_count(g.h) - n0
    lam_ms, lam_n = pg.jagp_profile_read(g.h)
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    g.close()
    n, nd = sysm.n_up, sysm.n_dn
    flops = 2.0 * L * L * W * (n + nd)  # the two lambda-product launches: 2 L^2 per orbital row
    achieved = flops * args.force_steps / (lam_ms / 1e3) / 1e12 if lam_ms > 0 else None
    return {"metric": "E_L+forces/s", "value": W * ws * args.force_steps / (ms_max / 1e3), "unit": "configurations/s",
            "ms_per_step": ms_max / args.force_steps, "steps": args.force_steps, "warmup": args.force_warmup,
            "dtype": "f64", "workload": FORCES_WORKLOAD, "walkers_per_gpu": W, "gpu_launches": launches,
            "roofline": {"kernel": "k_lambda_rows (adjoint orbital rows)", "bound": "alu", "achieved": achieved,
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS if achieved else None, "traffic": None,
                         "launches": lam_n, "share_of_step": lam_ms / ms if ms > 0 else None}}


BATCH_WORKLOAD = ("batched uneven systems, mixed precision: 64 independent neutral He systems, N uniform in "
                  "{8,...,128} (N/2 up, N/2 down, N/2 atoms), 16 Gaussians/atom, 512 walkers per system, every sweep "
                  "one replay of a captured CUDA graph over all systems; FP64 refresh of G^-1 every 16 moves of a "
                  "spin half-sweep and at its end")


def batch_bench(pg, torch, dist, args, dev, rank, ws):
    """Walker-electron moves/s of the batched mixed-precision path."""
    import synth
    systems = synth.config3_systems(seed=0, n_systems=args.batch_systems)
    W = args.batch_walkers
    members, pos, tunings = [], [], []
    for s in systems:
        m = pg.JAGP(s, W, seed=0, precision=pg.JAGP_PREC_MIXED, refresh_moves=16)
        p = m.positions(synth.init_walkers(s, W * ws, seed=0)[rank * W:(rank + 1) * W])
        m.eval(p)
        if not NO_AUTOTUNE:
            tunings.append(m.autotune(p))  # per system, before the graph is captured
        members.append(m)
        pos.append(p)
    b = pg.Batch(members, pos, walker0=[rank * W] * len(members), n_streams=args.batch_streams)
    b.sweep(args.warmup, sweep0=0)
    torch.cuda.synchronize()
    b.acc.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("batched")
    e0.record()
    b.sweep(args.batch_sweeps, sweep0=args.warmup)
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    bits = 0
    for m in members:
        bits |= m.status()
    acc = b.acc.cpu().numpy()
    b.close()
    for m in members:
        m.close()
    moves = W * sum(s.N for s in systems) * args.batch_sweeps * ws
    return {"metric": "walker-electron moves/s", "value": moves / (ms_max / 1e3), "unit": "walker-electron moves/s",
            "ms_per_sweep": ms_max / args.batch_sweeps, "sweeps": args.batch_sweeps, "warmup": args.warmup,
            "systems": len(systems), "walkers_per_system": W, "moves_per_sweep": moves // args.batch_sweeps // ws,
            "acceptance": float(acc[:, 2].sum()) / (moves / ws), "status_bits": bits,
            "dtype": "f32+bf16 (f64 refresh)", "workload": BATCH_WORKLOAD,
            "tuning": tuning_summary(tunings)}


def tuning_summary(tunings):
    """How often each tile choice won among the autotuned handles (None without tuning)."""
    if not tunings:
        return None
    keys = ("tile_proposals", "tile_refresh", "umma_bn_left", "umma_bn_right", "umma_stages_left",
            "umma_stages_right")
    out = {"handles": len(tunings)}
    for k in keys:
        counts = {}
        for t in tunings:
            counts[str(t[k])] = counts.get(str(t[k]), 0) + 1
        out[k] = counts
    return out


LARGE_WORKLOAD = ("large system, mixed precision: 256 He atoms in a 26 bohr cube (min separation 1.5), N=512 "
                  "(256 up, 256 down), 16 s/p/d Gaussians/atom (L=4096), banded lambda (|i-j| <= 204) stored dense, "
                  "J1 + J2, 1024 walkers/GPU; FP64 refresh of G^-1 every N_up moves, e_L every sweep")


def large_bench(pg, torch, dist, args, dev, rank, ws, local):
    """Walker-electron moves/s of the mixed path on the 512-electron system
    (G^-1 in global memory, in-place Gauss-Jordan refresh, tiled kernels)."""
    import numpy as np
    import synth
    sysm = synth.config5()
    W = args.large_walkers
    x0 = np.ascontiguousarray(synth.init_walkers(sysm, W * ws, seed=0)[rank * W:(rank + 1) * W])
    rr = timed_sweeps(pg, torch, dist, sysm, W, rank * W, x0, pg.JAGP_PREC_MIXED, args.large_steps, 3, ws, dev,
                      local, pg.KERNEL_LAMBDA_ROWS, label="large",
                      pin=json.loads(args.large_tuning) if args.large_tuning else None)
    xs = rr["r"][:args.large_force_walkers].clone()
    rr["g"].close()
    forces = large_forces(pg, torch, dist, sysm, xs, ws, dev) if args.large_force_walkers > 0 else None
    N, L = sysm.N, sysm.L
    kp = (L + 63) // 64 * 64
    secs = rr["prof_ms"] / 1e3
    issued = fixed_pairs(sysm) * 2.0 * kp * L * rr["accepted"]
    tc = issued / secs / 1e12 if secs > 0 else None
    return {"metric": "walker-electron moves/s", "value": W * N * args.large_steps * ws / (rr["ms_max"] / 1e3),
            "unit": "walker-electron moves/s", "ms_per_sweep": rr["ms_max"] / args.large_steps,
            "sweeps": args.large_steps, "warmup": 3, "walkers_per_gpu": W,
            "acceptance": rr["accepted"] / (W * N * args.large_steps), "status_bits": rr["bits"],
            "gpu_launches": rr["launches"], "dtype": "f32+bf16 (f64 refresh)", "workload": LARGE_WORKLOAD,
            "clocks": rr["clocks"], "tuning": rr["tuning"],
            "roofline": {"kernel": "k_umma_gemm (tcgen05, BF16 fixed-point slices)", "bound": "tensor",
                         "achieved": tc, "peak": BF16_SUSTAINED_TFLOPS, "unit": "TFLOP/s",
                         "frac": tc / BF16_SUSTAINED_TFLOPS if tc else None, "traffic": None,
                         "peak_source": BF16_PEAK_SOURCE,
                         "launches": rr["prof_n"], "share_of_step": rr["prof_ms"] / rr["ms"] if rr["ms"] > 0 else None},
            "forces": forces}


def large_forces(pg, torch, dist, sysm, xs, ws, dev):
    """E_L + forces per second on the 512-electron system (FP64 adjoint): the
    sampled walkers' configurations, one jagp_eval + jagp_grad per step."""
    W = xs.shape[0]
    g = pg.JAGP(sysm, W, seed=0)
    r = xs.contiguous()

    def step():
        g.eval(r)
        eL = g.local_energy(r)
        sL = 2.0 * (eL - eL.mean()) / W
        sE = torch.full((W,), 1.0 / W, dtype=torch.float64, device=dev)
        return g.grad(r, seed_logpsi=sL, seed_eL=sE)
    step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.nvtx.range_push("large_forces")
    e0.record()
    step()
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    g.close()
    return {"metric": "E_L+forces/s", "value": W * ws / (float(t.item()) / 1e3), "unit": "configurations/s",
            "ms_per_step": float(t.item()), "walkers_per_gpu": W, "dtype": "f64",
            "note": "one jagp_eval + local_energy + jagp_grad (FP64) on configurations of the mixed sweeps"}


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2002_07401_gb300 as pg
    import synth
    from paper_2002_07401_gb300 import shard

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the CPU oracle is not a fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)

    if args.large_only:
        # the 512-electron measurement alone (for profiling its launches)
        large = large_bench(pg, torch, dist, args, dev, rank, ws, local)
        if rank == 0:
            emit(dict(large, n_gpus=ws, higher_is_better=True, scaling="weak", data="synthetic"))
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    sysm = synth.config2()
    W = args.walkers
    N, L = sysm.N, sysm.L
    x_all = synth.init_walkers(sysm, W * ws, seed=0)
    walker0 = shard.walker_offset(W, rank)
    x0 = np.ascontiguousarray(x_all[walker0:walker0 + W])
    mixed_primary = args.precision == "mixed"
    prec = pg.JAGP_PREC_MIXED if mixed_primary else pg.JAGP_PREC_FP64

    run = timed_sweeps(pg, torch, dist, sysm, W, walker0, x0, prec, args.steps, args.warmup, ws, dev, local,
                       pg.KERNEL_LAMBDA_ROWS)
    g, r, eL = run["g"], run["r"], run["eL"]
    h = g.h

    # end to end through the public API with host buffers: pinned host positions
    # in, e_L and positions out, every step (state rebuilt by jagp_eval)
    hx = torch.from_numpy(x0.copy()).pin_memory()
    he = torch.empty(W, dtype=torch.float64).pin_memory()
    hr = torch.empty_like(hx).pin_memory()
    e2e_steps = max(2, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        r.copy_(hx, non_blocking=True)
        pg.jagp_eval(h, r, W, g.state)
        pg.vmc_sweep(h, r, g.state, W, 1, walker0, 10_000 + k, eL, None)
        he.copy_(eL[0], non_blocking=True)
        hr.copy_(r, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_value = W * N * e2e_steps * ws / float(e2e_t.item())
    g.close()

    # the other precision on the same workload, beside the primary
    other = None
    if not args.no_other:
        oprec = pg.JAGP_PREC_FP64 if mixed_primary else pg.JAGP_PREC_MIXED
        other = timed_sweeps(pg, torch, dist, sysm, W, walker0, x0, oprec, args.steps, args.warmup, ws, dev, local,
                             pg.KERNEL_LAMBDA_ROWS)
        other["g"].close()

    # FP64-equivalent lambda products on the tensor cores (fp64_tensor_cores=1)
    tc64 = None
    if not args.no_fp64tc:
        tc64 = timed_sweeps(pg, torch, dist, sysm, W, walker0, x0, pg.JAGP_PREC_FP64, args.steps, args.warmup, ws, dev,
                            local, pg.KERNEL_LAMBDA_ROWS, fp64_tc=True)
        tc64["g"].close()
    forces = None if args.no_forces else forces_bench(pg, torch, dist, args, dev, rank, ws, local)
    forces_tc = None
    if not args.no_forces and not args.no_fp64tc:
        forces_tc = forces_bench(pg, torch, dist, args, dev, rank, ws, local, fp64_tc=True)
        forces_tc["dtype"] = "f64 (lambda products FP64-equivalent on tensor cores)"
        forces_tc["roofline"] = None
    batched = None if args.no_batch else batch_bench(pg, torch, dist, args, dev, rank, ws)
    large = None if args.no_large else large_bench(pg, torch, dist, args, dev, rank, ws, local)

    if rank != 0:
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    def summary(rr, mixed):
        moves = W * N * args.steps * ws
        value = moves / (rr["ms_max"] / 1e3)
        flops = 2.0 * L * L * rr["accepted"]  # lambda products: 2 L^2 flops per accepted row
        secs = rr["prof_ms"] / 1e3
        achieved = flops / secs / 1e12 if secs > 0 else None
        d = {"value": value, "ms_per_step": rr["ms_max"] / args.steps,
             "el_per_s": W * args.steps * ws / (rr["ms_max"] / 1e3),
             "acceptance": rr["accepted"] / (W * N * args.steps), "status_bits": rr["bits"],
             "gpu_launches": rr["launches"], "clocks": rr["clocks"], "tuning": rr["tuning"]}
        if mixed:
            kp = (L + 63) // 64 * 64
            issued = fixed_pairs(sysm) * 2.0 * kp * L * rr["accepted"]  # BF16 slice-pair products per row
            tc = issued / secs / 1e12 if secs > 0 else None
            d["roofline"] = {"kernel": "k_umma_gemm (tcgen05, BF16 fixed-point slices)", "bound": "tensor",
                             "achieved": tc, "peak": BF16_SUSTAINED_TFLOPS, "unit": "TFLOP/s",
                             "frac": tc / BF16_SUSTAINED_TFLOPS if tc else None, "traffic": None,
                             "algorithmic_tflops": achieved, "peak_source": BF16_PEAK_SOURCE,
                             "launches": rr["prof_n"],
                             "avg_launch_ms": rr["prof_ms"] / max(rr["prof_n"], 1),
                             "share_of_step": rr["prof_ms"] / rr["ms"] if rr["ms"] > 0 else None}
        else:
            traffic_per_row, _ = profiled_traffic(kernel_source_hash())
            rows_per_launch = rr["accepted"] / max(rr["prof_n"], 1)
            d["roofline"] = {"kernel": "k_lambda_rows", "bound": "alu", "achieved": achieved,
                             "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
                             "traffic": traffic_per_row * rows_per_launch if traffic_per_row else None,
                             "peak_source": "nominal FP64 of GB300 (152 SM x 2 DFMA/clk x 2.07 GHz; "
                                            "measured register probe 1.19)",
                             "launches": rr["prof_n"], "avg_launch_ms": rr["prof_ms"] / max(rr["prof_n"], 1),
                             "share_of_step": rr["prof_ms"] / rr["ms"] if rr["ms"] > 0 else None}
        return d

    prim = summary(run, mixed_primary)
    out = {
        "metric": METRIC, "value": prim["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": prim["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+bf16 (f64 refresh)" if mixed_primary else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "walkers_per_gpu": W, "n_electrons": N, "basis_functions": L,
                   "precision": args.precision, "l2": "inputs larger than L2 (walker state ~1 GB per GPU)",
                   "parallelism": f"walker shards x{ws}"},
        "el_per_s": prim["el_per_s"], "acceptance": prim["acceptance"], "status_bits": prim["status_bits"],
        "roofline": prim["roofline"], "gpu_launches": prim["gpu_launches"], "tuning": prim["tuning"],
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(hx.numel() * 8),
                "d2h_bytes_per_step": int(he.numel() * 8 + hr.numel() * 8), "steps": e2e_steps},
        "clocks": prim["clocks"],
    }
    if other is not None:
        o = summary(other, not mixed_primary)
        o["precision"] = "fp64" if mixed_primary else "mixed"
        o["speedup_vs_primary"] = o["value"] / prim["value"]
        out["mixed" if not mixed_primary else "fp64"] = o
    if tc64 is not None:
        o = summary(tc64, False)
        kp = (L + 63) // 64 * 64
        nsl = 7 if L <= 512 else 8
        secs = tc64["prof_ms"] / 1e3
        issued = nsl * (nsl + 1) / 2 * 2.0 * kp * L * tc64["accepted"]
        tc = issued / secs / 1e12 if secs > 0 else None
        o["roofline"] = {"kernel": "k_umma_gemm (tcgen05, FP64-equivalent: %d BF16 slices, FP64 epilogue)" % nsl,
                         "bound": "tensor", "achieved": tc, "peak": BF16_SUSTAINED_TFLOPS, "unit": "TFLOP/s",
                         "frac": tc / BF16_SUSTAINED_TFLOPS if tc else None, "traffic": None,
                         "algorithmic_fp64_tflops": 2.0 * L * L * tc64["accepted"] / secs / 1e12 if secs > 0 else None,
                         "peak_source": BF16_PEAK_SOURCE,
                         "launches": tc64["prof_n"], "share_of_step": tc64["prof_ms"] / tc64["ms"] if tc64["ms"] else None}
        o["precision"] = "fp64 (lambda products FP64-equivalent on tensor cores)"
        o["speedup_vs_primary"] = o["value"] / prim["value"]
        out["fp64_tc"] = o
    if forces is not None:
        out["forces"] = forces
    if forces_tc is not None:
        out["forces_fp64tc"] = forces_tc
    if batched is not None:
        out["batched"] = batched
    if large is not None:
        out["large"] = large
    if ws == 1 and not args.no_cpu_baseline:
        mv, els, cores, sample, secs = oracle_rate(sysm, target_s=args.cpu_seconds)
        out["cpu_baseline"] = {"value": mv, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"{sample}; {secs:.1f} s; {cpu_model()}"}
    emit(out)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--walkers", type=int, default=4096)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-other", action="store_true", help="skip timing the other precision")
    ap.add_argument("--no-forces", action="store_true", help="skip the E_L + forces measurement")
    ap.add_argument("--no-fp64tc", action="store_true", help="skip the FP64-equivalent tensor-core measurement")
    ap.add_argument("--force-walkers", type=int, default=2048)
    ap.add_argument("--force-steps", type=int, default=2)
    ap.add_argument("--force-warmup", type=int, default=1)
    ap.add_argument("--no-batch", action="store_true", help="skip the batched uneven-systems measurement")
    ap.add_argument("--batch-systems", type=int, default=64)
    ap.add_argument("--batch-walkers", type=int, default=512)
    ap.add_argument("--batch-sweeps", type=int, default=20)
    ap.add_argument("--batch-streams", type=int, default=16)
    ap.add_argument("--no-large", action="store_true", help="skip the 512-electron mixed-precision measurement")
    ap.add_argument("--large-walkers", type=int, default=1024)
    ap.add_argument("--large-steps", type=int, default=3)
    ap.add_argument("--large-only", action="store_true", help="run only the 512-electron measurement")
    ap.add_argument("--large-tuning", default=None,
                    help="JSON tile choices for the 512-electron line (jagp_set_tuning) instead of autotuning")
    ap.add_argument("--large-force-walkers", type=int, default=16,
                    help="walkers of the 512-electron FP64 forces measurement (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-autotune", action="store_true", help="skip the tile autotuner (heuristic tiles)")
    args = ap.parse_args()
    global NO_AUTOTUNE
    NO_AUTOTUNE = args.no_autotune
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
