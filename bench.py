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
(fp64, mixed, fp64tc, batched, forces, large, large_forces, sr, lrdmc), so that a profiler
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


def _hbm_peak():
    """Measured HBM copy bandwidth (MEASURED_PEAKS.json), else the fallback 6.8 TB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            v = float(json.load(fh)["hbm_gbs"])
        if v > 0:
            return v, "measured HBM copy (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError, TypeError):
        pass
    return 6800.0, "fallback HBM 6.8 TB/s (no MEASURED_PEAKS file)"


HBM_GBS, HBM_SOURCE = _hbm_peak()


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
# BF16 slice-pair products per element of the mixed path's lambda products:
# both the up-spin rows (phi^T lambda) and the down-spin rows (lambda phi) take
# all 21 pairs of the six-slice operands (two-float results)
PAIRS_UP, PAIRS_DN = 21, 21
NO_AUTOTUNE = False  # --no-autotune: time the shape heuristics' tiles


def tensor_roofline(kernel, achieved, issued, launches, prof_ms, ms, work):
    """Roofline of a tensor-core kernel: `achieved` is the method's work
    (algorithmic flops) per second of kernel time, against the measured BF16
    peak; the issued BF16 slice-pair rate is reported beside it."""
    return {"kernel": kernel, "bound": "tensor", "achieved": achieved, "peak": BF16_SUSTAINED_TFLOPS,
            "unit": "TFLOP/s", "frac": achieved / BF16_SUSTAINED_TFLOPS if achieved else None, "traffic": None,
            "work": work, "issued_tflops": issued,
            "issued_frac": issued / BF16_SUSTAINED_TFLOPS if issued else None, "peak_source": BF16_PEAK_SOURCE,
            "launches": launches, "avg_launch_ms": prof_ms / max(launches, 1),
            "share_of_step": prof_ms / ms if ms > 0 else None}


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
def oracle_rate(sysm, target_s: float = 15.0, max_walkers: int = 4096, threads: int = 0):
    """Oracle VMC sweeps + local energies on a bounded sample of the same
    workload (up to all of its walkers, then more sweeps) sized to roughly
    target_s seconds, on all host cores (threads = 0) or the given number;
    returns (moves/s, e_L/s, cores, sample description, seconds)."""
    import oracle
    import synth
    o = oracle.Oracle(sysm)
    cores = threads if threads > 0 else oracle.max_threads()
    Ws, sweeps = max(cores, 8) if threads == 0 else 2, 1
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


# Arm CPU part numbers (/proc/cpuinfo "CPU part") of the cores these boxes may carry
ARM_PARTS = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1",
             "0xd49": "Arm Neoverse N2", "0xd84": "Arm Neoverse V3", "0xd8e": "Arm Neoverse N3"}


def cpu_model():
    """The host CPU's model name: lscpu's, else /proc/cpuinfo's model name, else
    the Arm core named from its part number."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                name = line.split(":", 1)[1].strip()
                if name and name != "-":
                    return name
    except Exception:
        pass
    part = None
    try:
        for line in open("/proc/cpuinfo"):
            low = line.lower()
            if low.startswith("model name"):
                return line.split(":", 1)[1].strip()
            if low.startswith("cpu part"):
                part = line.split(":", 1)[1].strip()
    except OSError:
        pass
    if part:
        return ARM_PARTS.get(part, f"Arm core part {part}")
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
    eL_steps = torch.empty((steps, W), dtype=torch.float64, device=dev)
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
            pg.vmc_sweep(h, r, g.state, W, 1, walker0, warmup + k, eL_steps[k:k + 1], acc_steps[k:k + 1])
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
    eL.copy_(eL_steps[-1:])
    return {"g": g, "r": r, "eL": eL, "eL_steps": eL_steps, "acc_steps": acc_steps, "ms": ms,
            "ms_max": float(t.item()), "launches": launches,
            "prof_ms": prof_ms, "prof_n": prof_n, "accepted": float(acc[:, 2].sum()), "bits": bits,
            "clocks": clk.summary(), "tuning": tuning}


FORCES_WORKLOAD = ("adjoint gradients: 64 He atoms in a 16 bohr cube, N=128 (64 up, 64 down), 24 s/p/d Gaussians/"
                   "atom (L=1536), 2048 walkers/GPU; per configuration e_L, the ionic force vector (Hellmann-Feynman "
                   "+ Pulay, Eq. forces:aad with the space-warp transformation), d log|Psi|/d lambda and "
                   "d log|Psi|/d b")


def forces_bench(pg, torch, dist, args, dev, rank, ws, local, fp64_tc=False, steps=None):
    """E_L + forces per second: one step = jagp_grad over all walkers with the
    force-estimator seeds (sE = 1/M, sL = 2 (e_L - <e_L>)/M from the walkers'
    local energies), producing e_L, dE/dR, d log|Psi|/d lambda and d/d b."""
    import numpy as np
    import synth
    steps = args.force_steps if steps is None else steps
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
               R=torch.empty((na, 3), **f64), Rw=torch.empty((W, na, 3), **f64),
               r=torch.empty((W, sysm.N, 3), **f64))

    def call():
        # adjoint with the force seeds, then the space warp (Eq. forces:aad with the warp's total derivatives)
        pg.jagp_grad(g.h, r, g.state, W, work, sL, sE, out["eL"], out["lam"], out["jas"], None, out["Rw"], out["r"])
        pg.jagp_space_warp(g.h, r, W, out["r"], out["Rw"], seed_logpsi=sL, dR=out["R"])
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
    for _ in range(steps):
        call()
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches = pg.jagp_launch_count(g.h) - n0
    lam_ms, lam_n = pg.jagp_profile_read(g.h)
    pg.jagp_profile(g.h, pg.KERNEL_LAMBDA_ROWS, False)
    ms = e0.elapsed_time(e1)
    # the energy alone on the same configurations (log|Psi| and e_L: what a VMC
    # energy evaluation costs), for the cost ratio of forces to energy
    ecall = lambda: (pg.jagp_eval(g.h, r, W, g.state), pg.local_energy(g.h, r, g.state, W, out["eL"]))  # noqa
    ecall()
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    esteps = max(3, steps // 4)
    e2.record()
    for _ in range(esteps):
        ecall()
    e3.record()
    torch.cuda.synchronize()
    ems = e2.elapsed_time(e3)
    t = torch.tensor([ms, ems], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max, ems_max = float(t[0].item()), float(t[1].item())
    g.close()
    n, nd = sysm.n_up, sysm.n_dn
    flops = 2.0 * L * L * W * (n + nd)  # the two lambda-product launches: 2 L^2 per orbital row
    achieved = flops * steps / (lam_ms / 1e3) / 1e12 if lam_ms > 0 else None
    if fp64_tc:
        kp = (L + 63) // 64 * 64
        nsl = 7 if L <= 512 else 8
        issued = achieved * (nsl * (nsl + 1) // 2) * kp / L if achieved else None
        roof = tensor_roofline("k_umma_gemm (tcgen05, FP64-equivalent adjoint lambda products, %d slices)" % nsl,
                               achieved, issued, lam_n, lam_ms, ms,
                               "2 L^2 FP64-equivalent flop per orbital row of the two adjoint lambda products")
    else:
        roof = {"kernel": "k_lambda_rows (adjoint orbital rows)", "bound": "alu", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS if achieved else None,
                "traffic": None, "work": "2 L^2 flop per orbital row of the two adjoint lambda products",
                "launches": lam_n, "share_of_step": lam_ms / ms if ms > 0 else None}
    return {"metric": "E_L+forces/s", "value": W * ws * steps / (ms_max / 1e3), "unit": "configurations/s",
            "ms_per_step": ms_max / steps, "steps": steps, "warmup": args.force_warmup,
            "dtype": "f64", "workload": FORCES_WORKLOAD, "walkers_per_gpu": W, "gpu_launches": launches,
            "energy_only": {"metric": "E_L/s", "value": W * ws * esteps / (ems_max / 1e3),
                            "unit": "configurations/s", "ms_per_step": ems_max / esteps, "steps": esteps,
                            "note": "jagp_eval + local_energy on the same configurations"},
            "forces_to_energy_cost": (ms_max / steps) / (ems_max / esteps) if ems_max > 0 else None,
            "roofline": roof}


REWEIGHTED_WORKLOAD = ("finite-variance forces on the adjoint workload's system (64 He, N=128, L=1536): walkers "
                       "sampled from the guiding function (theta = 3/8, eps tuned to <W> = 0.8), reweighting factors "
                       "W = (R / max(R, eps))^2, reweighted force seeds, adjoint and space warp")


def reweighted_forces_bench(pg, torch, dist, args, dev, rank, ws, local):
    """The full finite-variance force estimator of Sec. "Atomic forces": guided
    sampling (eps tuned so that <W> is near 0.8), the weights, the reweighted
    seeds, the FP64 adjoint and the space warp; one step = weights + seeds +
    adjoint + warp on all walkers."""
    import numpy as np
    import synth
    sysm = synth.config4()
    W = args.reweighted_walkers
    x0 = np.ascontiguousarray(synth.init_walkers(sysm, W * ws, seed=1)[rank * W:(rank + 1) * W])
    g = pg.JAGP(sysm, W, seed=1)
    r = g.positions(x0)
    g.eval(r)
    g.sweep(r, 4, walker0=rank * W, energies=False)
    eps = pg.tune_guiding_eps(g, r, target=0.8, rounds=6, sweeps=2, walker0=rank * W, sweep0=10)
    eL, _ = g.sweep(r, 2, walker0=rank * W, sweep0=100)
    e = eL[-1].contiguous()
    f64 = dict(dtype=torch.float64, device=dev)
    na = sysm.n_atoms
    wts = torch.empty(W, **f64)
    work = torch.empty(pg.jagp_grad_workspace_bytes(g.h, W), dtype=torch.uint8, device=dev)
    Rw, rb, dR = torch.empty((W, na, 3), **f64), torch.empty((W, sysm.N, 3), **f64), torch.empty((na, 3), **f64)
    jas = torch.empty(3, **f64)

    def step():
        pg.jagp_guiding_weights(g.h, g.state, W, 0.375, eps, weights=wts)
        sL, sE, mean = pg.jagp_force_seeds(e, wts)
        pg.jagp_grad(g.h, r, g.state, W, work, sL, sE, None, None, jas, None, Rw, rb)
        pg.jagp_space_warp(g.h, r, W, rb, Rw, seed_logpsi=sL, dR=dR)
        return mean
    step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.nvtx.range_push("forces_reweighted")
    e0.record()
    for _ in range(args.reweighted_steps):
        mean = step()
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    mw = float(mean[1].item())
    g.close()
    return {"metric": "E_L+forces/s", "value": W * ws * args.reweighted_steps / (ms / 1e3), "unit": "configurations/s",
            "ms_per_step": ms / args.reweighted_steps, "steps": args.reweighted_steps, "walkers_per_gpu": W,
            "eps": eps, "mean_weight": mw, "dtype": "f64", "workload": REWEIGHTED_WORKLOAD}


BATCH_WORKLOAD = ("batched uneven systems, mixed precision: 64 independent neutral He systems, N uniform in "
                  "{8,...,128} (N/2 up, N/2 down, N/2 atoms), 16 Gaussians/atom, 512 walkers per system, every sweep "
                  "one replay of a captured CUDA graph over all systems; FP64 refresh of G^-1 every 16 moves of a "
                  "spin half-sweep and at its end")


def batch_bench(pg, torch, dist, args, dev, rank, ws, precision=None, sweeps=None):
    """Walker-electron moves/s of the batched path (mixed precision unless
    given), then the roofline of its lambda products from one profiled sweep
    of every member outside the graph (CUDA events cannot sit inside it)."""
    import synth
    if precision is None:
        precision = pg.JAGP_PREC_MIXED
    mixed = precision == pg.JAGP_PREC_MIXED
    nsw = args.batch_sweeps if sweeps is None else sweeps
    systems = synth.config3_systems(seed=0, n_systems=args.batch_systems)
    W = args.batch_walkers
    members, pos, tunings = [], [], []
    for s in systems:
        m = pg.JAGP(s, W, seed=0, precision=precision, refresh_moves=16)
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
    torch.cuda.nvtx.range_push("batched" if mixed else "batched_fp64")
    e0.record()
    b.sweep(nsw, sweep0=args.warmup)
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
    launches_per_sweep = b.launches_per_sweep()
    b.close()
    # the other form of the same batched sweep (bit-identical results): grouped
    # launches (one per kernel and point of the sweep over all systems) beside
    # per-system launches over streams, or the reverse
    other = None
    other_sweeps = args.batch_grouped_sweeps if mixed else min(2, args.batch_grouped_sweeps)
    if other_sweeps > 0:
        ns_other = 0 if args.batch_streams > 0 else 16
        b2 = pg.Batch(members, pos, walker0=[rank * W] * len(members), n_streams=ns_other)
        b2.sweep(2, sweep0=nsw + args.warmup)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record()
        b2.sweep(other_sweeps, sweep0=nsw + args.warmup + 2)
        g1.record()
        torch.cuda.synchronize()
        gms = g0.elapsed_time(g1) / other_sweeps
        other = {"form": "grouped launches" if ns_other == 0 else "per-system launches over 16 streams",
                 "ms_per_sweep": gms, "value": W * sum(s.N for s in systems) / (gms / 1e3),
                 "unit": "walker-electron moves/s (one GPU)", "sweeps": other_sweeps,
                 "graph_launches_per_sweep": b2.launches_per_sweep()}
        b2.close()
    # roofline: every member's lambda products of one sweep, timed per launch
    lam_ms, lam_n, flops = 0.0, 0, 0.0
    acc1 = torch.empty((1, 4), dtype=torch.float64, device=dev)
    for s, m, p in zip(systems, members, pos):
        pg.jagp_profile(m.h, pg.KERNEL_LAMBDA_ROWS, True)
        pg.jagp_profile_read(m.h)
        pg.vmc_sweep(m.h, p, m.state, W, 1, rank * W, 100000, None, acc1)
        ms_k, n_k = pg.jagp_profile_read(m.h)
        pg.jagp_profile(m.h, pg.KERNEL_LAMBDA_ROWS, False)
        lam_ms += ms_k
        lam_n += n_k
        flops += 2.0 * s.L * s.L * float(acc1[0, 2].item())
    for m in members:
        m.close()
    achieved = flops / (lam_ms / 1e3) / 1e12 if lam_ms > 0 else None
    if mixed:
        roof = tensor_roofline("k_umma_gemm (tcgen05, BF16 fixed-point slices), all member systems", achieved,
                               achieved * PAIRS_UP if achieved else None, lam_n, lam_ms, 0.0,
                               "2 L^2 flop per accepted orbital row, summed over the systems of one sweep; issued: "
                               "%d BF16 slice-pair products per flop (before padding K to 64)" % PAIRS_UP)
    else:
        roof = {"kernel": "k_lambda_rows, all member systems", "bound": "alu", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS if achieved else None,
                "traffic": None, "work": "2 L^2 flop per accepted orbital row, summed over the systems of one sweep",
                "launches": lam_n, "avg_launch_ms": lam_ms / max(lam_n, 1)}
    roof["note"] = "kernel time from one profiled sweep of each member outside the graph"
    moves = W * sum(s.N for s in systems) * nsw * ws
    return {"metric": "walker-electron moves/s", "value": moves / (ms_max / 1e3), "unit": "walker-electron moves/s",
            "ms_per_sweep": ms_max / nsw, "sweeps": nsw, "warmup": args.warmup,
            "systems": len(systems), "walkers_per_system": W, "moves_per_sweep": moves // nsw // ws,
            "acceptance": float(acc[:, 2].sum()) / (moves / ws), "status_bits": bits,
            "dtype": "f32+bf16 (f64 refresh)" if mixed else "f64", "workload": BATCH_WORKLOAD if mixed else
            BATCH_WORKLOAD.replace("mixed precision", "plain FP64"), "graph_launches_per_sweep": launches_per_sweep,
            "form": "grouped launches" if args.batch_streams <= 0 else
            "per-system launches over %d streams" % args.batch_streams, "other_form": other,
            "tuning": tuning_summary(tunings), "roofline": roof}


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
            "roofline": tensor_roofline("k_umma_gemm (tcgen05, BF16 fixed-point slices)",
                                        2.0 * L * L * rr["accepted"] / secs / 1e12 if secs > 0 else None, tc,
                                        rr["prof_n"], rr["prof_ms"], rr["ms"],
                                        "2 L^2 flop per accepted orbital row (the lambda product); issued: %d BF16 "
                                        "slice-pair products per flop" % PAIRS_UP),
            "forces": forces}


PIPELINE_WORKLOAD = ("large system, full pipeline: the 512-electron system's 1024 walkers swept in mixed precision "
                     "(autotuned tiles), and every 10 sweeps the FP64 adjoint forces (lambda products FP64-equivalent "
                     "on the tensor cores) of a fixed subset of the walkers' current configurations: e_L, the ionic "
                     "force vector (Hellmann-Feynman + Pulay, Eq. forces:aad with the space warp), d log|Psi|/d lambda "
                     "and d/d b")


def pipeline_bench(pg, torch, dist, args, dev, rank, ws, local, pin=None):
    """Config 5 as one timed pipeline: args.pipeline_sweeps mixed sweeps of all
    walkers; after every args.pipeline_every sweeps the first
    args.pipeline_force_walkers walkers' configurations go (device to device)
    to an FP64 handle, which evaluates log|Psi|, e_L and the adjoint with the
    force-estimator seeds.  Moves/s counts every walker's moves over the whole
    region; E_L+forces/s counts the force configurations over the time of the
    force phases (CUDA events around them on the same stream)."""
    import numpy as np
    import synth
    sysm = synth.config5()
    W, K = args.large_walkers, args.pipeline_force_walkers
    S, every = args.pipeline_sweeps, args.pipeline_every
    x0 = np.ascontiguousarray(synth.init_walkers(sysm, W * ws, seed=0)[rank * W:(rank + 1) * W])
    gm = pg.JAGP(sysm, W, seed=0, precision=pg.JAGP_PREC_MIXED)
    if pin:  # the large line's choices for the same system and walker count
        gm.set_tuning(pin)
        tuning = pin
    else:
        tuning = None if NO_AUTOTUNE else gm.autotune()
    r = gm.positions(x0)
    gf = pg.JAGP(sysm, K, seed=0, fp64_tc=True)
    rf = torch.empty((K, sysm.N, 3), dtype=torch.float64, device=dev)
    work = torch.empty(pg.jagp_grad_workspace_bytes(gf.h, K), dtype=torch.uint8, device=dev)
    f64 = dict(dtype=torch.float64, device=dev)
    L, na = sysm.L, sysm.n_atoms
    eLf, lam = torch.empty(K, **f64), torch.empty((L, L), **f64)
    jas, dR = torch.empty(3, **f64), torch.empty((na, 3), **f64)
    eL = torch.empty((1, W), **f64)
    stream = torch.cuda.current_stream()

    Rw = torch.empty((K, na, 3), **f64)
    rb = torch.empty((K, sysm.N, 3), **f64)

    def forces():
        rf.copy_(r[:K])
        pg.jagp_eval(gf.h, rf, K, gf.state)
        pg.local_energy(gf.h, rf, gf.state, K, eLf)
        sL, sE, _ = pg.jagp_force_seeds(eLf)
        pg.jagp_grad(gf.h, rf, gf.state, K, work, sL, sE, eLf, lam, jas, None, Rw, rb)
        pg.jagp_space_warp(gf.h, rf, K, rb, Rw, seed_logpsi=sL, dR=dR)

    pg.jagp_eval(gm.h, r, W, gm.state)
    for k in range(3):
        pg.vmc_sweep(gm.h, r, gm.state, W, 1, rank * W, k, eL, None)
    forces()
    torch.cuda.synchronize()
    nforce = S // every
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nforce)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = pg.jagp_launch_count(gm.h) + pg.jagp_launch_count(gf.h)
    with ClockSampler(local) as clk:
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("pipeline")
        e0.record(stream)
        q = 0
        for t in range(S):
            pg.vmc_sweep(gm.h, r, gm.state, W, 1, rank * W, 3 + t, eL, None)
            if (t + 1) % every == 0:
                ev[q][0].record(stream)
                forces()
                ev[q][1].record(stream)
                q += 1
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
    launches = pg.jagp_launch_count(gm.h) + pg.jagp_launch_count(gf.h) - n0
    ms = e0.elapsed_time(e1)
    fms = sum(a.elapsed_time(b) for a, b in ev)
    t = torch.tensor([ms, fms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms, fms = float(t[0].item()), float(t[1].item())
    bits = gm.status() | gf.status()
    force_norm = float(dR.norm().item())
    gm.close()
    gf.close()
    return {"metric": "walker-electron moves/s", "value": W * sysm.N * S * ws / (ms / 1e3),
            "unit": "walker-electron moves/s", "ms_total": ms, "sweeps": S, "force_every": every,
            "force_evaluations": nforce, "force_walkers": K,
            "forces": {"metric": "E_L+forces/s", "value": K * nforce * ws / (fms / 1e3), "unit": "configurations/s",
                       "ms_per_evaluation": fms / max(nforce, 1)},
            "sweep_share": (ms - fms) / ms if ms > 0 else None, "status_bits": bits, "gpu_launches": launches,
            "dtype": "f32+bf16 sweeps (f64 refresh), f64 adjoint", "workload": PIPELINE_WORKLOAD,
            "walkers_per_gpu": W, "clocks": clk.summary(), "tuning": tuning, "last_force_norm": force_norm}


SR_WORKLOAD = ("stochastic reconfiguration on the C2 workload (16 He, N=32, L=320, 4096 walkers/GPU, after sweeps): "
               "per-walker log-derivatives of every lambda entry and the three Jastrow parameters (P = L^2 + 3 = "
               "102403), then the regularised step (eps = 1e-3) by matrix-free preconditioned CG")


def sr_bench(pg, torch, dist, args, dev, rank, ws, local):
    """SR steps per second: one step = jagp_logpsi_derivs (the M x P samples,
    FP64 per-walker products) + jagp_sr_step with a fixed number of CG
    iterations (each two passes over the samples, bound by HBM)."""
    import numpy as np
    import synth
    sysm = synth.config2()
    W = args.walkers
    P = sysm.L * sysm.L + 3
    x0 = np.ascontiguousarray(synth.init_walkers(sysm, W * ws, seed=0)[rank * W:(rank + 1) * W])
    g = pg.JAGP(sysm, W, seed=0)
    r = g.positions(x0)
    g.eval(r)
    g.sweep(r, 2, walker0=rank * W)
    eL = g.local_energy(r)
    O = torch.empty((W, P), dtype=torch.float64, device=dev)
    work = torch.empty(pg.jagp_sr_workspace_bytes(W, P), dtype=torch.uint8, device=dev)
    it = args.sr_iters
    g.logpsi_derivs(r, O)
    pg.jagp_sr_step(O, eL, eps=1e-3, delta=0.05, max_iter=it, tol=0.0, work=work)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    steps = args.sr_steps
    d_ms = cg_ms = 0.0
    if ws > 1:
        dist.barrier()
    torch.cuda.nvtx.range_push("sr")
    for _ in range(steps):
        ev[0].record()
        g.logpsi_derivs(r, O)
        ev[1].record()
        f, da, iters, res = pg.jagp_sr_step(O, eL, eps=1e-3, delta=0.05, max_iter=it, tol=0.0, work=work)
        ev[2].record()
        torch.cuda.synchronize()
        d_ms += ev[0].elapsed_time(ev[1])
        cg_ms += ev[1].elapsed_time(ev[2])
    torch.cuda.nvtx.range_pop()
    t = torch.tensor([d_ms, cg_ms], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    d_ms, cg_ms = float(t[0].item()), float(t[1].item())
    g.close()
    # the CG: two passes over the FP64 samples per iteration, plus the three of the set-up (Obar, diag S, f)
    cg_bytes = (2.0 * iters + 3.0) * W * P * 8
    gbs = cg_bytes / (cg_ms / steps / 1e3) / 1e9
    n, nd, L = sysm.n_up, sysm.n_dn, sysm.L
    dflops = 2.0 * W * (n * nd * L + n * L * L)
    return {"metric": "SR steps/s", "value": steps * ws / ((d_ms + cg_ms) / 1e3), "unit": "steps/s",
            "ms_per_step": (d_ms + cg_ms) / steps, "ms_log_derivs": d_ms / steps, "ms_solve": cg_ms / steps,
            "cg_iterations": iters, "relative_residual": res, "parameters": P, "samples_per_gpu": W, "dtype": "f64",
            "workload": SR_WORKLOAD,
            "roofline": {"kernel": "SR solve (k_sr_rowdot + k_sr_colsum passes over the samples)", "bound": "hbm",
                         "achieved": gbs, "peak": HBM_GBS, "unit": "GB/s", "frac": gbs / HBM_GBS, "traffic": None,
                         "work": "(2 iterations + 3) x M x P x 8 bytes of samples read", "peak_source": HBM_SOURCE},
            "log_derivs_roofline": {"kernel": "k_bgemm_tn (per-walker FP64 products)", "bound": "alu",
                                    "achieved": dflops / (d_ms / steps / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                                    "unit": "TFLOP/s",
                                    "frac": dflops / (d_ms / steps / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
                                    "work": "2 (N_up N_dn L + N_up L^2) flop per walker"}}


LRDMC_WORKLOAD = ("lattice-regularised DMC on the C2 workload (16 He, N=32, L=320, 4096 walkers/GPU, FP64), "
                  "continuous time, fixed node: lattice a = 0.2 bohr, gamma = 0, projection tau = 0.01 /Ha per "
                  "generation, reconfiguration after each generation")


def lrdmc_bench(pg, torch, dist, args, dev, rank, ws, local):
    """LRDMC hops/s: one step = one generation (a continuous-time projection
    of length tau, every walker hopping until its time is spent, then the
    reconfiguration).  Each round of hops recomputes the moved rows' lambda
    products, and G~^{-1}, the kinetic vectors M and e_L of the walkers that
    moved, and the 6N hop ratios of every walker still moving."""
    import numpy as np
    import synth
    sysm = synth.config2()
    W = args.walkers
    a, gamma, tau = 0.2, 0.0, 0.01
    x0 = np.ascontiguousarray(synth.init_walkers(sysm, W * ws, seed=0)[rank * W:(rank + 1) * W])
    g = pg.JAGP(sysm, W, seed=0)
    r = g.positions(x0)
    g.eval(r)
    g.sweep(r, 4, walker0=rank * W, energies=False)
    e_ref = float(g.local_energy(r).mean().item())
    work = torch.empty(pg.jagp_lrdmc_workspace_bytes(g.h, W), dtype=torch.uint8, device=dev)
    w = torch.ones(W, dtype=torch.float64, device=dev)
    eL = torch.empty(W, dtype=torch.float64, device=dev)
    hops = torch.empty(W, dtype=torch.int32, device=dev)
    flags = torch.empty(W, dtype=torch.int32, device=dev)
    stats = torch.empty(2, dtype=torch.float64, device=dev)
    parent = torch.empty(W, dtype=torch.int32, device=dev)

    def generation(gen):
        pg.jagp_lrdmc_project(g.h, r, g.state, W, work, w, gen, a, gamma, tau, e_ref, 1 << 20, rank * W, eL, hops,
                              flags)
        h = hops.sum()
        hm = hops.max()
        pg.jagp_lrdmc_branch(g.h, r, W, work, w, eL, gen, parent, stats)
        return h, hm

    for gen in range(args.lrdmc_warmup):
        generation(gen)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = pg.jagp_launch_count(g.h)
    tot_h, rounds, ebar = 0, 0, []
    if ws > 1:
        dist.barrier()
    torch.cuda.nvtx.range_push("lrdmc")
    ev0.record()
    for k in range(args.lrdmc_gens):
        h, hm = generation(args.lrdmc_warmup + k)
        tot_h += int(h.item())
        rounds += int(hm.item()) + 1
        ebar.append(float(stats[1].item()))
    ev1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    ms = ev0.elapsed_time(ev1)
    launches = pg.jagp_launch_count(g.h) - n0
    t = torch.tensor([ms, tot_h], dtype=torch.float64, device=dev)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t[0].item())
    g.close()
    K = args.lrdmc_gens
    n, nd, N, L = sysm.n_up, sysm.n_dn, sysm.N, sysm.L
    # dense FP64 work per hop: the moved row's lambda product (2 L^2), the
    # refresh product G~ = Phi_up Bt^T (2 n^2 L) and the kinetic vectors M
    # (2 N n L) of the walker that moved; per walker and round it is active
    # (its hops plus its last round): the 6N hop-ratio dots (12 N L)
    flops = tot_h * (2.0 * L * L + 2.0 * n * n * L + 2.0 * N * n * L) + (tot_h + W * K) * 12.0 * N * L
    tf = flops / (ms / 1e3) / 1e12
    return {"metric": "LRDMC walker hops/s", "value": tot_h * ws / (ms / 1e3), "unit": "walker hops/s",
            "ms_per_generation": ms / K, "generations": K, "warmup": args.lrdmc_warmup,
            "hops_per_walker_per_generation": tot_h / (W * K), "rounds_per_generation": rounds / K,
            "ebar": ebar, "e_ref": e_ref, "gpu_launches": launches, "dtype": "f64", "workload": LRDMC_WORKLOAD,
            "roofline": {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": tf / FP64_PEAK_TFLOPS,
                         "work": "per hop 2 L^2 (lambda row) + 2 N_up^2 L (G~) + 2 N N_up L (M); per active "
                                 "walker and round 12 N L (hop ratios); over the whole generation",
                         "peak_source": "nominal FP64 of GB300 (152 SM x 2 DFMA/clk x 2.07 GHz)"}}


C1_WORKLOAD = ("plain FP64 VMC, 4 H atoms in a 3 bohr cube, N=4 (2 up, 2 down), 6 s+p Gaussians/atom (L=24), "
               "spin-independent J2, no J1, 256 walkers/GPU")


def c1_bench(pg, torch, dist, args, dev, rank, ws, local):
    """The smallest configuration: launch- and latency-bound (a few microseconds
    of work per kernel), reported as moves/s only."""
    import numpy as np
    import synth
    sysm = synth.config1()
    W = 256
    x0 = np.ascontiguousarray(synth.init_walkers(sysm, W * ws, seed=0)[rank * W:(rank + 1) * W])
    rr = timed_sweeps(pg, torch, dist, sysm, W, rank * W, x0, pg.JAGP_PREC_FP64, args.c1_sweeps, args.warmup, ws,
                      dev, local, pg.KERNEL_LAMBDA_ROWS, label="c1")
    rr["g"].close()
    ms = rr["ms_max"]
    # the same sweeps replayed as one captured CUDA graph per sweep (a one-system
    # batch: the sweep index comes from a device counter), which removes the
    # host's launch cost from every kernel
    g = pg.JAGP(sysm, W, seed=0)
    p = g.positions(x0)
    g.eval(p)
    b = pg.Batch([g], [p], walker0=[rank * W], n_streams=1)
    b.sweep(args.warmup, sweep0=0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b.sweep(args.c1_sweeps, sweep0=args.warmup)
    e1.record()
    torch.cuda.synchronize()
    gms = e0.elapsed_time(e1)
    graph = {"ms_per_sweep": gms / args.c1_sweeps, "value": W * sysm.N * args.c1_sweeps / (gms / 1e3),
             "unit": "walker-electron moves/s (one GPU)", "graph_launches_per_sweep": b.launches_per_sweep(),
             "note": "one CUDA graph replay per sweep (jagp_batch over this one system)"}
    b.close()
    g.close()
    return {"metric": "walker-electron moves/s", "value": W * sysm.N * args.c1_sweeps * ws / (ms / 1e3),
            "unit": "walker-electron moves/s", "ms_per_sweep": ms / args.c1_sweeps, "sweeps": args.c1_sweeps,
            "gpu_launches": rr["launches"], "launches_per_sweep": rr["launches"] / args.c1_sweeps,
            "us_per_launch": ms * 1e3 / max(rr["launches"], 1), "graph": graph, "dtype": "f64",
            "workload": C1_WORKLOAD,
            "roofline": {"bound": "latency", "note": "each launch carries microseconds of work: the sweep is bound "
                         "by launch latency and the sequential acceptance, not by a roofline", "frac": None}}


def reblocked_energy(pg, eL_steps, acc_steps, ws, dev):
    """VMC energy of the timed sweeps: the reblocked mean and error bar of this
    rank's samples (jagp_reblock), and the sums over all ranks' accumulators
    (the only collective of the data path: one all-reduce per statistics block)."""
    from paper_2002_07401_gb300 import shard
    levels, stats = pg.jagp_reblock(eL_steps)
    st = stats.cpu().numpy()
    tot = shard.sum_over_ranks(acc_steps[:, :3].sum(dim=0), device=dev).cpu().numpy()
    T, W = eL_steps.shape
    return {"mean": float(st[0]), "error": float(st[1]), "block_level": int(st[2]), "plateau": bool(st[3]),
            "levels": int(levels.shape[0]), "samples": T * W,
            "all_ranks_mean": float(tot[0] / (T * W * ws)),
            "all_ranks_sum_eL2": float(tot[1]), "all_ranks_accepted": float(tot[2])}


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
    energy = reblocked_energy(pg, run["eL_steps"], run["acc_steps"], ws, dev)

    # end to end through the public API with host buffers: pinned host positions
    # in, e_L and positions out, every step (state rebuilt by jagp_eval)
    hx = torch.from_numpy(x0.copy()).pin_memory()
    he = torch.empty(W, dtype=torch.float64).pin_memory()
    hr = torch.empty_like(hx).pin_memory()
    e2e_steps = max(2, args.steps)
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
        forces_tc = forces_bench(pg, torch, dist, args, dev, rank, ws, local, fp64_tc=True,
                                 steps=args.force_tc_steps)
        forces_tc["dtype"] = "f64 (lambda products FP64-equivalent on tensor cores)"
    batched = None if args.no_batch else batch_bench(pg, torch, dist, args, dev, rank, ws)
    batched64 = None
    if not args.no_batch and not args.no_other:
        batched64 = batch_bench(pg, torch, dist, args, dev, rank, ws, precision=pg.JAGP_PREC_FP64,
                                sweeps=args.batch_fp64_sweeps)
    large = None if args.no_large else large_bench(pg, torch, dist, args, dev, rank, ws, local)
    pipeline = None if args.no_large else pipeline_bench(pg, torch, dist, args, dev, rank, ws, local,
                                                         pin=large.get("tuning") if large else None)
    sr = None if args.no_sr else sr_bench(pg, torch, dist, args, dev, rank, ws, local)
    lrdmc = None if args.no_lrdmc else lrdmc_bench(pg, torch, dist, args, dev, rank, ws, local)
    reweighted = None if args.no_forces else reweighted_forces_bench(pg, torch, dist, args, dev, rank, ws, local)
    c1 = None if args.no_c1 else c1_bench(pg, torch, dist, args, dev, rank, ws, local)

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
            d["roofline"] = tensor_roofline("k_umma_gemm (tcgen05, BF16 fixed-point slices)", achieved, tc,
                                            rr["prof_n"], rr["prof_ms"], rr["ms"],
                                            "2 L^2 flop per accepted orbital row (the lambda product); issued: "
                                            "%d BF16 slice-pair products per flop on K padded to 64" % PAIRS_UP)
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
        o["roofline"] = tensor_roofline(
            "k_umma_gemm (tcgen05, FP64-equivalent: %d BF16 slices, FP64 epilogue)" % nsl,
            2.0 * L * L * tc64["accepted"] / secs / 1e12 if secs > 0 else None, tc, tc64["prof_n"], tc64["prof_ms"],
            tc64["ms"], "2 L^2 FP64-equivalent flop per accepted orbital row; issued: %d BF16 slice-pair products "
            "per flop on K padded to 64" % (nsl * (nsl + 1) // 2))
        o["precision"] = "fp64 (lambda products FP64-equivalent on tensor cores)"
        o["speedup_vs_primary"] = o["value"] / prim["value"]
        out["fp64_tc"] = o
    if forces is not None:
        out["forces"] = forces
    if forces_tc is not None:
        out["forces_fp64tc"] = forces_tc
    if batched is not None:
        out["batched"] = batched
    if batched64 is not None:
        out["batched_fp64"] = batched64
    if large is not None:
        out["large"] = large
    if pipeline is not None:
        out["pipeline"] = pipeline
    if sr is not None:
        out["sr"] = sr
    if lrdmc is not None:
        out["lrdmc"] = lrdmc
    if reweighted is not None:
        out["forces_reweighted"] = reweighted
    if c1 is not None:
        out["c1"] = c1
    out["energy"] = energy
    if ws == 1 and not args.no_cpu_baseline:
        mv, els, cores, sample, secs = oracle_rate(sysm, target_s=args.cpu_seconds)
        mv1, _, _, sample1, secs1 = oracle_rate(sysm, target_s=args.cpu_seconds / 3, threads=1)
        out["cpu_baseline"] = {"value": mv, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"{sample}; {secs:.1f} s; {cpu_model()}", "cpu_model": cpu_model(),
                               "single_thread": {"value": mv1, "unit": UNIT, "cores": 1,
                                                 "sample": f"{sample1}; {secs1:.1f} s"}}
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
    ap.add_argument("--force-steps", type=int, default=20)
    ap.add_argument("--force-warmup", type=int, default=1)
    ap.add_argument("--force-tc-steps", type=int, default=8)
    ap.add_argument("--reweighted-walkers", type=int, default=512)
    ap.add_argument("--reweighted-steps", type=int, default=5)
    ap.add_argument("--no-batch", action="store_true", help="skip the batched uneven-systems measurement")
    ap.add_argument("--batch-systems", type=int, default=64)
    ap.add_argument("--batch-walkers", type=int, default=512)
    ap.add_argument("--batch-sweeps", type=int, default=50)
    ap.add_argument("--batch-fp64-sweeps", type=int, default=5)
    ap.add_argument("--batch-streams", type=int, default=16,
                    help="> 0: per-system launches over that many streams; 0 (or -k): grouped launches over all "
                         "systems (in k lanes)")
    ap.add_argument("--batch-grouped-sweeps", type=int, default=10,
                    help="sweeps of the other batched form (grouped launches, or per-system streams) timed beside")
    ap.add_argument("--no-large", action="store_true", help="skip the 512-electron mixed-precision measurement")
    ap.add_argument("--large-walkers", type=int, default=1024)
    ap.add_argument("--large-steps", type=int, default=20)
    ap.add_argument("--pipeline-sweeps", type=int, default=20)
    ap.add_argument("--pipeline-every", type=int, default=10)
    ap.add_argument("--pipeline-force-walkers", type=int, default=64)
    ap.add_argument("--no-sr", action="store_true", help="skip the stochastic-reconfiguration measurement")
    ap.add_argument("--sr-steps", type=int, default=3)
    ap.add_argument("--sr-iters", type=int, default=50)
    ap.add_argument("--no-c1", action="store_true", help="skip the 4-electron latency-bound line")
    ap.add_argument("--no-lrdmc", action="store_true", help="skip the lattice-regularised DMC measurement")
    ap.add_argument("--lrdmc-gens", type=int, default=3)
    ap.add_argument("--lrdmc-warmup", type=int, default=1)
    ap.add_argument("--c1-sweeps", type=int, default=200)
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
