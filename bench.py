#!/usr/bin/env python
"""Benchmark of one RVEA generation (the whole hot path) on GB300.

A step is one generation: reproduction + evaluation, selection, finalize
(+ reference-vector adaptation and gamma every round(f_r t_max) generations).
Default workload: DTLZ1, m = 3, d = 5000, N = NV = 9870 (H = 139), the
large-scale configuration.  The metric is generations per second; the
roofline entry reports the reproduction kernel against the measured HBM copy
bandwidth.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica (the path
has no exchange step): value = all generations of all ranks / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RVEA generations/s & HBM GB/s vs roofline (plain vs batched); serve p50/p99"

WORKLOADS = {
    "dtlz1_m3_d5000_N9870": dict(m=3, d=5000, N=9870, H=139, problem=1, t_max=1000),
    "dtlz2_m3_d12_N105": dict(m=3, d=12, N=105, H=13, problem=0, t_max=100),
    "dtlz3_m3_d5000_N9870": dict(m=3, d=5000, N=9870, H=139, problem=3, t_max=1000),
    "dtlz4_m3_d5000_N9870": dict(m=3, d=5000, N=9870, H=139, problem=4, t_max=1000),
    # the extensibility experiment's reproduction operators (Sec. 4.4) on the
    # large-scale configuration: DE/rand/1/bin, random reproduction, CSO
    "de_dtlz1_m3_d5000_N9870": dict(m=3, d=5000, N=9870, H=139, problem=1, t_max=1000,
                                    reproduction=1, de_F=0.5, de_CR=0.9),
    "random_dtlz1_m3_d5000_N9870": dict(m=3, d=5000, N=9870, H=139, problem=1, t_max=1000,
                                        reproduction=2),
    "cso_dtlz1_m3_d5000_N9870": dict(m=3, d=5000, N=9870, H=139, problem=1, t_max=1000,
                                     reproduction=3, cso_phi=0.1),
    "pso_dtlz1_m3_d5000_N9870": dict(m=3, d=5000, N=9870, H=139, problem=1, t_max=1000,
                                     reproduction=4, pso_w=0.7298, pso_c1=1.49618,
                                     pso_c2=1.49618),
}
OPS = {0: "k_repro (mating + SBX + g-terms; mutation and evaluation in k_mutate when d > 1024)",
       1: "k_repro_de (DE/rand/1/bin: four rows read, one child row written, evaluation)",
       2: "k_repro_rand (random reproduction: one child row written, evaluation)",
       3: "k_cso_mean + k_cso_centre + k_repro_cso (CSO: swarm centre over the valid rows; "
          "winner, loser and loser velocity rows read, child row and velocity written; "
          "evaluation)",
       4: "k_repro_pso (PSO: particle, its velocity and personal best, leader rows read; child "
          "row, velocity and personal best written; evaluation)"}
COMMON = dict(alpha=2.0, f_r=0.1, eta_c=20.0, eta_m=20.0, p_c=1.0, p_m=1.0)


def max_over_ranks(x: float, dist, device) -> float:
    """The maximum of x over the ranks of the process group (x if none): a
    replica run is as slow as its slowest rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, steps: int, ms_max: float) -> float:
    """Whole-job generations/s of `world` replicas of `steps` generations each,
    timed by the slowest rank."""
    return world * steps / (ms_max * 1e-3)


def repro_bytes(wl) -> int:
    """Algorithmic bytes of one generation's reproduction, d float32 per row
    (objectives are O(N m)).  SBX: read 2*ceil(N/2) parent rows, write N
    child rows.  DE/rand/1/bin: read four rows (target, r1, r2, r3), write one,
    per offspring.  Random: write N rows.  CSO: read the winner's and loser's
    rows and the loser's velocity, write the child's row and velocity, per
    offspring, plus (phi > 0) one pass over the valid rows for the centre,
    counted as N rows (all slots valid).  PSO: read the particle's row,
    velocity and personal best and the leader's row, write the child's row,
    velocity and personal best, per offspring."""
    N, d, op = wl["N"], wl["d"], wl.get("reproduction", 0)
    if op == 1:
        return 5 * N * d * 4
    if op == 2:
        return N * d * 4
    if op == 3:
        return (5 + (1 if wl.get("cso_phi", 0.0) > 0 else 0)) * N * d * 4
    if op == 4:
        return 7 * N * d * 4
    P = (N + 1) // 2
    return (2 * P + N) * d * 4


def run_config(args, wl, world):
    """The config of a single-run workload's line, the same for both arms."""
    return {"workload": args.workload, **wl, **COMMON,
            "parallelism": f"replicas x{world}",
            "l2": f"no flush: {2 * wl['N'] * wl['d'] * 4 / 1e6:.0f} MB moved per generation "
                  f"> 129 MB L2 (inputs larger than L2)"}


def oracle_params(orc, wl, seed=0):
    """The oracle's parameters of a bench workload (its operator included)."""
    extra = {}
    if wl.get("reproduction", 0):
        extra = dict(op=wl["reproduction"], de_F=wl.get("de_F", 0.5), de_CR=wl.get("de_CR", 0.9),
                     cso_phi=wl.get("cso_phi", 0.0), pso_w=wl.get("pso_w", 0.7298),
                     pso_c1=wl.get("pso_c1", 1.49618), pso_c2=wl.get("pso_c2", 1.49618))
    return orc.make_params(m=wl["m"], d=wl["d"], N=wl["N"], H=wl["H"], problem=wl["problem"],
                           t_max=wl["t_max"], seed=seed, **COMMON, **extra)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        return float(mp["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_sha() -> str:
    h = hashlib.sha256()
    for f in ("k_repro.cu", "rvea_device.cuh", "eval_steps.cuh"):
        with open(os.path.join(ROOT, "paper_2404_01159_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str):
    """DRAM bytes per reproduction launch from the committed ncu summary, if it
    was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", f"k_repro_{workload}.txt")
    if not os.path.exists(path):
        return None
    sha, traffic = None, None
    with open(path) as f:
        for line in f:
            if line.startswith("source_sha:"):
                sha = line.split(":", 1)[1].strip()
            if line.startswith("dram_bytes_per_launch:"):
                traffic = float(line.split(":", 1)[1].strip())
    return traffic if sha == source_sha() else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.rows = []
        self.ok = False
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100",
                                       "-i", gpu_id], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
            return
        self.first = threading.Event()
        self.live = False
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        self.first.wait(timeout=10)
        self.ok = True

    def _read(self):
        for line in self.p.stdout:
            self.first.set()
            if self.live:
                self.rows.append([x.strip() for x in line.split(",")])

    def start(self):
        self.live = True

    def stop(self):
        self.live = False
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(self.rows)}


def cpu_baseline(wl, seconds=20.0):
    """The FP64 oracle, as it stands, on the host cores: whole generations of
    the same workload from a seeded initial population, as many as fit in
    about `seconds` (at least one)."""
    from oracle import oracle as orc
    cores = os.cpu_count() or 1
    orc.set_threads(cores)
    p = oracle_params(orc, wl)
    V0, st = orc.initial_state(p)
    n = 0
    t0 = time.perf_counter()
    while True:
        orc.generation(p, V0, st)
        n += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "generations/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} whole FP64 oracle generation(s) of the same workload, "
                      f"{dt:.1f} s on {cores} host threads (OpenMP over rows)"}


def run_reference(args, wl, rank, world):
    if rank != 0:
        return
    from oracle import oracle as orc
    cores = os.cpu_count() or 1
    orc.set_threads(cores)
    p = oracle_params(orc, wl)
    V0, st = orc.initial_state(p)
    W = min(args.warmup, 20)   # untimed, bounded: the oracle needs no warming
    for _ in range(W):
        orc.generation(p, V0, st)
    budget = 150.0
    n = 0
    t0 = time.perf_counter()
    while n < args.steps:
        orc.generation(p, V0, st)
        n += 1
        if time.perf_counter() - t0 > budget:
            break
    dt = time.perf_counter() - t0
    v = n / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "generations/s",
            "n_gpus": 0, "steps": n, "warmup": W, "ms_per_step": 1e3 * dt / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Philox initial population, closed-form objective)",
            "config": run_config(args, wl, 1),
            "generations": f"t = {W + 1}..{W + n}",
            "cpu_baseline": {"value": v, "unit": "generations/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{n} of the requested {args.steps} generations "
                                       f"(bounded to ~{budget:.0f} s), FP64 oracle"},
            "e2e": {"value": v, "unit": "generations/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


BATCHED = "batched256_uneven"


def batch_bytes(insts) -> int:
    """Algorithmic bytes of one batched generation: every run's parents read
    (2 ceil(N/2) rows) and children written (N rows)."""
    return sum((2 * ((i.N + 1) // 2) + i.N) * i.d * 4 for i in insts)


def main_batched(args, rank, world, local, emit=True, steps=None, warmup=None, with_cpu=True):
    """Uneven runs stepped together: one CUDA graph per batched generation,
    plans from the autotuner; the same runs stepped one after another is the
    sequential comparison.  Returns the JSON line (printed when emit)."""
    import torch
    torch.cuda.set_device(local)
    from paper_2404_01159_gb300 import Batch, Run, autotune
    from paper_2404_01159_gb300.workloads import batched_set
    K = args.steps if steps is None else steps
    W = max(3, args.warmup if warmup is None else warmup)
    insts = batched_set(args.batched_runs, 500, seed0=rank * args.batched_runs)
    t0 = time.perf_counter()
    runs = [Run(**i.run_kwargs()) for i in insts]
    torch.cuda.synchronize()
    t_init = time.perf_counter() - t0
    t0 = time.perf_counter()
    plans = [autotune(r) for r in runs]
    t_tune = time.perf_counter() - t0
    batch = Batch(runs)
    batch.step(W)
    torch.cuda.synchronize()
    props = torch.cuda.get_device_properties(local)
    gid = str(getattr(props, "uuid", "")) or str(local)
    if gid and not gid.startswith("GPU-") and len(gid) >= 32:
        gid = "GPU-" + gid
    sampler = ClockSampler(gid) if rank == 0 else None
    if sampler:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    batch.step(K)
    e1.record()
    e1.synchronize()
    if sampler:
        sampler.stop()
    ms = e0.elapsed_time(e1)
    for r in runs:
        r.sync_status()
    # the same runs, one after another (each its own graph), K_seq generations each
    Ks = max(3, min(K, 10))
    for r in runs:
        r.step(2)
    torch.cuda.synchronize()
    e0.record()
    for r in runs:
        r.step(Ks)
    e1.record()
    e1.synchronize()
    ms_seq = e0.elapsed_time(e1)
    Kp = max(1, min(K, 20))
    phases = batch.step_profiled(Kp)
    launches_per_step = batch.launches_per_step()
    batch.free()
    nb = batch_bytes(insts)
    hbm_peak, peak_kind = peaks()
    value = len(runs) * K / (ms * 1e-3)
    seq = len(runs) * Ks / (ms_seq * 1e-3)
    achieved = nb / (ms / K * 1e-3) / 1e9
    modes = {}
    for pl in plans:
        key = ("pruned-smem", "pruned-L1", "fused-tail")[pl["sel_mode"] - 1] if pl["sel_mode"] else \
            f"scan/{pl['sel_per_sm']}"
        key += "+staged" if pl["repro_staged"] else "+direct"
        modes[key] = modes.get(key, 0) + 1
    cpu = None
    if world == 1 and not args.no_cpu_baseline and with_cpu:
        cpu = cpu_baseline_batched(insts, args.cpu_seconds)
    for r in runs:
        r.free()
    if rank != 0:
        return None
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "run-generations/s",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": ms / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (256 seeded uneven runs, closed-form DTLZ objectives)",
        "config": {"workload": BATCHED, "runs": len(runs),
                   "m": "uniform {2,3,5,10}", "N": f"{min(i.N for i in insts)}..{max(i.N for i in insts)}",
                   "d": f"{min(i.d for i in insts)}..{max(i.d for i in insts)} log-uniform",
                   "t_max": 500, **{k: v for k, v in COMMON.items()},
                   "workspace_gb": sum(r.workspace_nbytes for r in runs) / 1e9,
                   "parallelism": "one CUDA graph per batched generation",
                   "l2": f"no flush: {nb / 1e9:.1f} GB moved per batched generation > 129 MB L2",
                   "plans": modes},
        "sequential": {"value": seq, "unit": "run-generations/s", "steps_per_run": Ks,
                       "what": "the same runs stepped one after another (rvea_step, "
                               "graph per run)"},
        "batched_over_sequential": value / seq,
        "roofline": {"kernel": "whole batched generation (all phases of all runs)",
                     "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "peak_kind": peak_kind, "traffic": None,
                     "algorithmic_bytes_per_launch": nb,
                     "avg_launch_ms": ms / K,
                     "timing": f"CUDA events around {K} graph replays"},
        "phase_ms_per_generation": {"repro": phases[0] / Kp, "select_pruned": phases[1] / Kp,
                                    "select_scan": phases[2] / Kp, "finalize": phases[3] / Kp,
                                    "gamma_tiles": phases[4] / Kp},
        "setup_s": {"init": t_init, "autotune": t_tune},
        "cpu_baseline": cpu,
        "e2e": None,
        "gpu_launches": K * launches_per_step,
        "clocks": sampler.summary() if sampler else None,
    }
    if emit:
        print(json.dumps(line), flush=True)
    return line


SERVE = "serve_poisson200"
NEURO = "neuro100x100_steps1000"


def main_neuro(args, rank, world, local):
    """Neuroevolution: 100 runs x 100 MLP policies (17-64-64-6, d = 5702),
    each child evaluated by a 1000-step rollout of the synthetic linear
    dynamics, stepped together as one CUDA graph per batched generation."""
    import torch
    torch.cuda.set_device(local)
    from paper_2404_01159_gb300 import NEURO_LINEAR, Batch, Run, autotune
    from paper_2404_01159_gb300.workloads import neuro_dynamics, policy_size
    K, W = args.steps, max(3, args.warmup)
    dyn = neuro_dynamics(0)
    d = policy_size()
    n_runs, N, H, t_max = 100, 100, 99, 100
    kw = dict(m=2, d=d, N=N, H=H, problem=NEURO_LINEAR, t_max=t_max, alpha=2.0, f_r=0.1,
              eta_c=20.0, eta_m=20.0, p_c=1.0, p_m=1.0)
    Kp = max(1, min(K, 5))

    def timed(gemv, sample, **op):
        """K batched generations of the 100 runs with the given GEMV form (and
        reproduction operator): (ms, per-phase ms, launches per step, clock
        summary)."""
        runs = [Run(seed=rank * n_runs + q, neuro=dict(dyn, gemv=gemv), **kw, **op)
                for q in range(n_runs)]
        for r in runs:
            autotune(r)
        batch = Batch(runs)
        batch.step(W)
        torch.cuda.synchronize()
        sampler = None
        if sample:
            props = torch.cuda.get_device_properties(local)
            gid = str(getattr(props, "uuid", "")) or str(local)
            if gid and not gid.startswith("GPU-") and len(gid) >= 32:
                gid = "GPU-" + gid
            sampler = ClockSampler(gid)
            sampler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        batch.step(K)
        e1.record()
        e1.synchronize()
        if sampler:   # the same loop, untimed, so that the clock record has samples
            t_soak = time.perf_counter()
            while time.perf_counter() - t_soak < args.soak_seconds:
                batch.step(K)
                torch.cuda.synchronize()
            sampler.stop()
        ms = e0.elapsed_time(e1)
        phases = batch.step_profiled(Kp)
        lps = batch.launches_per_step()
        for r in runs:
            r.sync_status()
        batch.free()
        return ms, phases, lps, (sampler.summary() if sampler else None)

    # the form the workload runs in: the policy GEMVs in FP32 on the CUDA
    # cores (gemv = 1, hidden-layer weights register-resident); the BF16
    # tensor-core form (gemv = 0) is timed beside it as the comparison
    ms, phases, launches_per_step, clocks = timed(1, rank == 0)
    ms16, ph16, _, _ = timed(0, False)
    # the same runs reproduced by CSO (the swarm the paper's neuroevolution
    # experiment picks), phi = 0.1
    ms_cso, ph_cso, _, _ = timed(1, False, reproduction=3, cso_phi=0.1)
    steps = dyn["steps"]
    gemm_flop = n_runs * N * steps * 2 * (64 * 17 + 64 * 64 + 6 * 64)
    eval_ms = phases[0] / Kp
    tf_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"] \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1900.0
    # FP32 CUDA-core peak: 152 SMs x 128 FMA/clock x 2 flop x 2.07 GHz
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    achieved = gemm_flop / (eval_ms * 1e-3) / 1e12
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_neuro(kw, dyn, args.cpu_seconds)
    if rank != 0:
        return
    line = {
        "metric": METRIC,
        "value": n_runs * K / (ms * 1e-3),
        "unit": "run-generations/s",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": ms / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 GEMV (CUDA cores), f32 dynamics",
        "data": "synthetic (seeded policies N(0, 0.1), seeded linear dynamics, rho(A) = 0.95)",
        "config": {"workload": NEURO, "runs": n_runs, "policies_per_run": N, "d": d,
                   "mlp": "17-64-64-6 tanh", "rollout_steps": steps, "sigma": dyn["sigma"],
                   "t_max": t_max, "m": 2, "H": H, "gemv": 1,
                   "l2": "rollouts are compute-bound; weights stay on chip for 1000 steps",
                   "parallelism": "one CUDA graph per batched generation"},
        "policies_per_s": n_runs * N * K / (ms * 1e-3),
        "bf16_tensor_cores": {
            "value": n_runs * K / (ms16 * 1e-3), "unit": "run-generations/s",
            "ms_per_step": ms16 / K,
            "rollout_ms": ph16[0] / Kp,
            "gemm_tflops": gemm_flop / (ph16[0] / Kp * 1e-3) / 1e12,
            "frac_of_bf16_peak": gemm_flop / (ph16[0] / Kp * 1e-3) / 1e12 / tf_peak,
            "fp32_speedup_over_this": ms16 / ms,
            "what": "the same workload with the policy GEMVs on the tensor cores (mma.sync "
                    "BF16 hi/lo operands, FP32 accumulate, rvea_neuro_dynamics.gemv = 0)"},
        "roofline": {"kernel": "k_rollout_f32 (1000-step rollout of every child)", "bound": "alu",
                     "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak,
                     "peak_kind": "derived: FP32 FMA rate, 152 SMs x 128 lanes x 2 flop x 2.07 GHz",
                     "traffic": None, "algorithmic_flop_per_launch": gemm_flop,
                     "avg_launch_ms": eval_ms,
                     "what": "useful policy-GEMM flops (2 x 5568 MAC per step per policy) over "
                             "the reproduction+rollout phase"},
        "phase_ms_per_generation": {"repro_rollout": phases[0] / Kp,
                                    "select_pruned": phases[1] / Kp,
                                    "select_scan": phases[2] / Kp, "finalize": phases[3] / Kp,
                                    "gamma_tiles": phases[4] / Kp},
        "cpu_baseline": cpu,
        "e2e": None,
        "gpu_launches": K * launches_per_step,
        "clocks": clocks,
        "cso": {"value": n_runs * K / (ms_cso * 1e-3), "unit": "run-generations/s",
                "ms_per_step": ms_cso / K, "repro_rollout_ms": ph_cso[0] / Kp,
                "what": "the same runs reproduced by CSO (phi = 0.1: swarm centre, "
                        "competitions, learning), the children evaluated by the FP32 rollout"},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_neuro(kw, dyn, seconds=20.0):
    """The FP64 oracle on the host cores: whole generations (100 rollouts of
    1000 steps each) of the first runs of the same workload."""
    from oracle import oracle as orc
    orc.build()
    threads = os.cpu_count() or 1
    orc.set_threads(threads)
    nd = orc.NeuroData(dyn["A"], dyn["B"], steps=dyn["steps"], sigma=dyn["sigma"])
    gens, t0 = 0, time.perf_counter()
    q = 0
    while time.perf_counter() - t0 < seconds:
        p = orc.make_params(m=2, d=kw["d"], N=kw["N"], H=kw["H"], problem=orc.NEURO,
                            t_max=kw["t_max"], L=-1.0, U=1.0, seed=q)
        V0, st = orc.initial_state(p, nd)
        orc.generation(p, V0, st, nd)
        gens += 1
        q += 1
    el = time.perf_counter() - t0
    return {"value": gens / el, "unit": "run-generations/s", "cores": threads, "kind": "oracle",
            "sample": f"{gens} run(s): initial population rollouts plus one generation each "
                      f"(FP64, 100 policies x 1000 steps per rollout set), initialisation in "
                      f"the time"}


def main_serve(args, rank, world, local, emit=True, rate=None, seconds=None, drain=None):
    """Serving: Poisson arrivals of runs (m, d, N, budget drawn per request),
    admitted by an HBM budget, their generations batched across live runs
    each step; time-to-result from arrival to the step that finished it.
    Returns the JSON line (printed when emit)."""
    import torch
    torch.cuda.set_device(local)
    from paper_2404_01159_gb300 import Server
    from paper_2404_01159_gb300.workloads import request_stream
    rate = args.serve_rate if rate is None else rate
    seconds = args.serve_seconds if seconds is None else seconds
    drain = args.serve_drain_seconds if drain is None else drain
    reqs = request_stream(rate, seconds, seed=rank)
    budget = int(args.serve_budget_gb * 1e9)
    srv = Server(budget, max_live=args.serve_max_live, autotune=True)
    props = torch.cuda.get_device_properties(local)
    gid = str(getattr(props, "uuid", "")) or str(local)
    if gid and not gid.startswith("GPU-") and len(gid) >= 32:
        gid = "GPU-" + gid
    sampler = ClockSampler(gid) if rank == 0 else None
    if sampler:
        sampler.start()
    arrival, budget_of, lat = {}, {}, []
    k, steps, gens_done, live_sum = 0, 0, 0, 0
    cap_s = seconds + drain
    outstanding = 0
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        while k < len(reqs) and reqs[k][0] <= now:
            at, inst = reqs[k]
            rid = srv.submit(inst.m, inst.d, inst.N, inst.H, inst.problem, inst.generations,
                             seed=inst.seed)
            arrival[rid], budget_of[rid] = at, inst.generations
            k += 1
            outstanding += 1
        if outstanding == 0:
            if k >= len(reqs):
                break
            time.sleep(max(0.0, min(0.01, reqs[k][0] - now)))
            continue
        st = srv.step()
        torch.cuda.current_stream().synchronize()
        steps += 1
        live_sum += st["live"]
        tdone = time.perf_counter() - t0
        for rid in srv.poll():
            srv.fetch(rid)
            lat.append(tdone - arrival.pop(rid))
            gens_done += budget_of.pop(rid)
            outstanding -= 1
        if tdone > cap_s:
            break
    wall = time.perf_counter() - t0
    if sampler:
        sampler.stop()
    srv.free()
    if rank != 0:
        return None
    lat.sort()
    pct = (lambda q: lat[min(len(lat) - 1, int(q * len(lat)))] if lat else None)
    line = {
        "metric": METRIC,
        "value": gens_done / wall,
        "unit": "run-generations/s",
        "n_gpus": world,
        "steps": steps,
        "warmup": 0,
        "ms_per_step": wall / max(1, steps) * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded Poisson request stream, closed-form DTLZ objectives)",
        "config": {"workload": SERVE, "rate_per_s": rate,
                   "arrivals_s": seconds, "requests": len(reqs),
                   "hbm_budget_gb": args.serve_budget_gb, "max_live": args.serve_max_live,
                   "m": "uniform {2,3,5,10}", "N": "100..9870", "d": "30..5000 log-uniform",
                   "generations": "U{50..1000}", **COMMON},
        "serve": {"completed": len(lat), "submitted": k, "unfinished": outstanding,
                  "p50_s": pct(0.50), "p99_s": pct(0.99), "mean_live_runs": live_sum / max(1, steps),
                  "wall_s": wall,
                  "what": "time-to-result = end of the step that finished the run - arrival; "
                          "wall-clock, the loop synchronises after every step"},
        "roofline": None,
        "cpu_baseline": None,
        "e2e": None,
        "gpu_launches": None,
        "clocks": sampler.summary() if sampler else None,
    }
    if emit:
        print(json.dumps(line), flush=True)
    return line


def sub_batched(args, local):
    """The batched form inside the default line: 256 uneven runs, a few graph
    replays, against the same runs stepped one after another."""
    try:
        b = main_batched(args, 0, 1, local, emit=False, steps=10, warmup=3, with_cpu=False)
        return {"workload": BATCHED, "value": b["value"], "unit": b["unit"],
                "ms_per_step": b["ms_per_step"], "steps": b["steps"],
                "sequential": b["sequential"]["value"],
                "batched_over_sequential": b["batched_over_sequential"],
                "roofline_frac": b["roofline"]["frac"], "gpu_launches": b["gpu_launches"],
                "phase_ms_per_generation": b["phase_ms_per_generation"],
                "setup_s": b["setup_s"], "clocks": b["clocks"]}
    except Exception as e:   # the headline line must survive
        return {"workload": BATCHED, "error": repr(e)[:300]}


def sub_serve(args, local, rates=(50.0, 200.0), seconds=8.0, drain=40.0):
    """The served form inside the default line: a short Poisson window at a
    rate below capacity and at the configuration's 200 requests/s."""
    out = {"workload": SERVE, "arrivals_s": seconds, "hbm_budget_gb": args.serve_budget_gb,
           "rates": []}
    for rate in rates:
        try:
            sv = main_serve(args, 0, 1, local, emit=False, rate=rate, seconds=seconds, drain=drain)
            out["rates"].append({"rate_per_s": rate, "value": sv["value"], "unit": sv["unit"],
                                 "p50_s": sv["serve"]["p50_s"], "p99_s": sv["serve"]["p99_s"],
                                 "completed": sv["serve"]["completed"],
                                 "submitted": sv["serve"]["submitted"],
                                 "mean_live_runs": sv["serve"]["mean_live_runs"],
                                 "wall_s": sv["serve"]["wall_s"], "clocks": sv["clocks"]})
        except Exception as e:
            out["rates"].append({"rate_per_s": rate, "error": repr(e)[:300]})
    return out


SWEEPS = {
    # the paper's speed sweeps (Sec. 4.1): population sizes 2^5 .. 2^14 at
    # d = 100, and dimensions 2^9 .. 2^18 at n = 100; DTLZ1, m = 3, 100
    # generations.  A size that is not a lattice size runs on the largest
    # Das-Dennis lattice with at most that many points (rvea_lattice_for).
    "sweep_pop_d100": dict(axis="n", points=[2 ** k for k in range(5, 15)], d=100, n=None),
    "sweep_dim_n100": dict(axis="d", points=[2 ** k for k in range(9, 19)], d=None, n=100),
}


def main_sweep(args, rank, world, local, name):
    """One line for a whole sweep: per point the GPU time per generation
    (CUDA events around 100 generations after a warm-up), achieved bytes per
    second of the reproduction against the HBM copy rate, and the FP64
    oracle's time per generation on the host cores over a bounded sample."""
    import torch
    torch.cuda.set_device(local)
    from paper_2404_01159_gb300 import Run, lattice_for, lattice_size
    sw = SWEEPS[name]
    hbm_peak, peak_kind = peaks()
    K, W = max(args.steps, 100), max(3, args.warmup)
    cores = os.cpu_count() or 1
    pts, cpu_left = [], args.cpu_seconds
    for x in sw["points"]:
        n = x if sw["axis"] == "n" else sw["n"]
        d = x if sw["axis"] == "d" else sw["d"]
        H = lattice_for(3, n)
        N = lattice_size(3, H)
        kw = dict(m=3, d=d, N=N, H=H, problem=1, t_max=100, **COMMON)
        run = Run(seed=11, **kw)
        run.step(W)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run.step(K)
        e1.record()
        e1.synchronize()
        run.sync_status()
        ms = e0.elapsed_time(e1) / K
        wl = dict(m=3, d=d, N=N)
        gbs = repro_bytes(wl) / (ms * 1e-3) / 1e9
        pt = {"n_requested": n, "N": N, "H": H, "d": d, "ms_per_generation": ms,
              "generations_per_s": 1e3 / ms, "whole_generation_gbs": gbs,
              "whole_generation_frac": gbs / hbm_peak}
        del run
        if world == 1 and not args.no_cpu_baseline and cpu_left > 0:
            from oracle import oracle as orc
            orc.set_threads(cores)
            p = orc.make_params(m=3, d=d, N=N, H=H, problem=1, t_max=100, seed=11, **COMMON)
            V0, st = orc.initial_state(p)
            t0, g = time.perf_counter(), 0
            while g < 3 and (g == 0 or time.perf_counter() - t0 < 2.0):
                orc.generation(p, V0, st)
                g += 1
            dt = (time.perf_counter() - t0) / g
            cpu_left -= time.perf_counter() - t0
            pt["oracle_s_per_generation"] = dt
            pt["gpu_over_oracle"] = dt / (ms * 1e-3)
        pts.append(pt)
    if rank != 0:
        return
    last = pts[-1]
    line = {
        "metric": METRIC, "value": last["generations_per_s"], "unit": "generations/s",
        "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": last["ms_per_generation"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Philox initial population, closed-form DTLZ1)",
        "config": {"workload": name, "axis": sw["axis"], "m": 3, "problem": "DTLZ1",
                   "generations_timed": K, **COMMON,
                   "l2": "no flush between generations (the small points fit in L2; "
                         "their throughput is launch- and latency-bound, as in the paper)"},
        "points": pts,
        "roofline": {"kernel": "whole generation at the last point", "bound": "hbm",
                     "achieved": last["whole_generation_gbs"], "peak": hbm_peak, "unit": "GB/s",
                     "frac": last["whole_generation_frac"], "peak_kind": peak_kind,
                     "traffic": None},
        "cpu_baseline": {"kind": "oracle", "cores": cores,
                         "sample": "up to 3 FP64 oracle generations per point, bounded"},
        "e2e": None,
        "gpu_launches": None,
        "clocks": None,
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_batched(insts, seconds=20.0):
    """The FP64 oracle on the host cores over a bounded sample of the same
    runs: one generation each of as many runs (in order) as fit in
    `seconds`."""
    from oracle import oracle as orc
    orc.build()
    threads = os.cpu_count() or 1
    orc.set_threads(threads)
    done, gens, t0 = 0, 0, time.perf_counter()
    for i in insts:
        p = orc.make_params(**i.run_kwargs())
        V0, st = orc.initial_state(p)
        orc.generation(p, V0, st)
        gens += 1
        done += 1
        if time.perf_counter() - t0 > seconds:
            break
    el = time.perf_counter() - t0
    return {"value": gens / el, "unit": "run-generations/s", "cores": threads, "kind": "oracle",
            "sample": f"one FP64 oracle generation (after its initialisation) of each of the "
                      f"first {done} runs of the same set, initialisation included in the time"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dtlz1_m3_d5000_N9870",
                    choices=sorted(WORKLOADS) + [BATCHED, SERVE, NEURO] + sorted(SWEEPS))
    ap.add_argument("--serve-rate", type=float, default=200.0, help="requests per second")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="arrival window")
    ap.add_argument("--serve-drain-seconds", type=float, default=60.0,
                    help="time allowed after the arrival window")
    ap.add_argument("--serve-budget-gb", type=float, default=80.0)
    ap.add_argument("--serve-max-live", type=int, default=320)
    ap.add_argument("--batched-runs", type=int, default=256,
                    help="runs of the batched workload (256; fewer only to profile a smaller case)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end pass")
    ap.add_argument("--e2e-generations", type=int, default=1000,
                    help="generations of the end-to-end pass (at least --steps)")
    ap.add_argument("--soak-seconds", type=float, default=1.5,
                    help="untimed run after the timed region, under the clock sampler")
    ap.add_argument("--no-sub", action="store_true",
                    help="omit the batched and served sub-results of the default line")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload in SWEEPS:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the oracle arm times the single-run workload; the sweep line "
                              "carries the oracle's time per point"}))
            return
        main_sweep(args, rank, world, local, args.workload)
        return
    if args.workload == NEURO:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the oracle arm times the single-run workload only"}))
            return
        main_neuro(args, rank, world, local)
        return
    if args.workload == SERVE:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the oracle arm times the single-run workload only"}))
            return
        main_serve(args, rank, world, local)
        return
    if args.workload == BATCHED:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the oracle arm times the single-run workload only"}))
            return
        main_batched(args, rank, world, local)
        return
    wl = WORKLOADS[args.workload]

    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2404_01159_gb300 import Run
    from paper_2404_01159_gb300._native import lib
    lib()

    K, W = args.steps, max(3, args.warmup)
    kw = dict(wl, **COMMON)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident throughput (graph replays) -------------------------
    run = Run(seed=1000 + rank, **kw)
    run.step(W)
    torch.cuda.synchronize()
    t_first = run.t
    props = torch.cuda.get_device_properties(local)
    gid = str(getattr(props, "uuid", "")) or str(local)
    if gid and not gid.startswith("GPU-") and len(gid) >= 32:
        gid = "GPU-" + gid
    sampler = ClockSampler(gid) if rank == 0 else None
    barrier()
    if sampler:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    run.step(K)
    e1.record()
    e1.synchronize()
    # untimed soak of the same generation loop, so that the clock sampler sees
    # the GPU under this load (the timed region alone is a few milliseconds)
    t_soak = time.perf_counter()
    while time.perf_counter() - t_soak < args.soak_seconds:
        run.step(200)
        torch.cuda.synchronize()
    soak_s = time.perf_counter() - t_soak
    if sampler:
        sampler.stop()
    barrier()
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, dist, "cuda")
    run.sync_status()
    from paper_2404_01159_gb300 import get_plan
    plan_mode = get_plan(run)["sel_mode"]
    p_adapt = max(1, int(kw["f_r"] * kw["t_max"] + 0.5))
    n_adapt = sum(1 for t in range(t_first, t_first + K) if t % p_adapt == 0)
    launches = (K - n_adapt) * run.launches_per_generation(False) + \
        n_adapt * run.launches_per_generation(True)
    del run

    # ---- per-kernel device time (CUDA events around every launch) -----------
    Kp = min(K, 500)
    prun = Run(seed=2000 + rank, **kw)
    prun.step(W)
    phases = prun.step_profiled(Kp)
    prun.sync_status()
    del prun
    repro_ms = phases[0] / Kp
    bytes_rep = repro_bytes(wl)
    hbm_peak, peak_kind = peaks()
    achieved = bytes_rep / (repro_ms * 1e-3) / 1e9

    # ---- end to end through the public API, host buffers --------------------
    N, m, d = wl["N"], wl["m"], wl["d"]
    Ke = max(K, args.e2e_generations)
    e2e_s = None
    if not args.no_e2e:
        hF = torch.empty((N, m), dtype=torch.float32, pin_memory=True)
        hV = torch.empty(N, dtype=torch.uint8, pin_memory=True)
        hX = torch.empty((N, d), dtype=torch.float32, pin_memory=True)
        barrier()
        t0 = time.perf_counter()
        erun = Run(seed=3000 + rank, **kw)            # host config -> device state
        for _ in range(Ke):
            erun.step(1)
            erun.objectives(hF, hV)                  # per-generation result to host
        erun.population(hX, hV)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e_s = max_over_ranks(e2e_s, dist, "cuda")
        erun.sync_status()
        del erun
    h2d_init = N * m * 8 * 2 + N * 16 + 4096       # lattice (f64 x2), float copy, tables
    d2h = Ke * (N * m * 4 + N) + N * d * 4 + N

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, args.cpu_seconds)
    value = replica_value(world, K, ms)
    clocks = sampler.summary() if sampler else None
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "generations/s",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": ms / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded Philox initial population, closed-form DTLZ objective)",
        "config": run_config(args, wl, world),
        "generations": f"t = {t_first}..{t_first + K - 1}",
        "roofline": {"kernel": OPS[wl.get("reproduction", 0)], "bound": "hbm",
                     "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                     "traffic": profiled_traffic(args.workload),
                     "algorithmic_bytes_per_launch": bytes_rep,
                     "avg_launch_ms": repro_ms,
                     "timing": f"CUDA events around each launch, {Kp} generations"},
        "phase_ms_per_generation": (
            {"repro": phases[0] / Kp,
             "tail_fused": phases[1] / Kp,
             "gamma_tiles_grid": phases[3] / Kp,
             "what": "tail_fused: mutation/evaluation, association and finalize in one "
                     "persistent launch"}
            if plan_mode == 3 else
            {"repro": phases[0] / Kp, "mutate_eval": phases[4] / Kp,
             "select": phases[1] / Kp, "finalize": phases[2] / Kp,
             "gamma_tiles_grid": phases[3] / Kp}),
        "plan": plan_mode,
        "whole_generation_hbm_gbs": bytes_rep / (ms / K * 1e-3) / 1e9,
        "whole_generation_frac": bytes_rep / (ms / K * 1e-3) / 1e9 / hbm_peak,
        "cpu_baseline": cpu,
        "e2e": None if e2e_s is None else {
            "value": world * Ke / e2e_s, "unit": "generations/s",
            "h2d_bytes_per_step": h2d_init / Ke, "d2h_bytes_per_step": d2h / Ke,
            "generations": Ke,
            "what": "init from host config + per-generation objectives to pinned host "
                    "+ final population to pinned host, over max(steps, 1000) generations"},
        "gpu_launches": launches,
        "clocks": None if clocks is None else dict(
            clocks, window=f"timed region + {soak_s:.1f} s untimed soak of the same loop"),
    }
    if world == 1 and not args.no_sub:
        line["batched"] = sub_batched(args, local)
        line["serve"] = sub_serve(args, local)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
