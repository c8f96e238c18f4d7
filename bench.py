#!/usr/bin/env python
"""GLD throughput on one GB300: particle-steps/s of the 262144-particle,
m_max = 400 suspension (FP32 history ring of 1.26 GB, larger than L2).

One step = the whole hot path: history convolution, pair dissipative force
and position update, cell-list rebuild, conservative force and velocity
update, VACF accumulation, and the colored-noise block every 64 steps.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead.
Under torchrun each rank steps an independent replica (different seed); there
is no data-path collective, only a barrier and a max over ranks of the time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLD particle-steps/s at N=262k,m_max=400"
UNIT = "particle-steps/s"
PROFILES = os.path.join(ROOT, "profiles")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4096)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gld", choices=["gld", "reference"])
    ap.add_argument("--workload", default="gld_n262144_m400")
    ap.add_argument("--profile-steps", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--hist", default="f32", choices=["f32", "bf16"])
    ap.add_argument("--kahan", action="store_true")
    ap.add_argument("--reference-seconds", type=float, default=120.0)
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def init_replicas(world: int, local: int, backend: str):
    """One process per GPU, each stepping an independent replica: the process
    group only carries the barrier and the max of the timings (no data-path
    collective)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value: float, world: int, device: str = "cpu") -> float:
    """The slowest rank's value (whole-job time is set by the last replica)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(n_per_rank: int, steps: int, world: int, ms_max: float) -> float:
    """Whole-job particle-steps/s: all ranks' particles over the slowest time."""
    return world * n_per_rank * steps / (ms_max / 1e3)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str, path: str):
        self.path, self.proc = path, None
        try:
            self.fh = open(path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", gpu_index, "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], None, set()
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_hash() -> str:
    src = os.path.join(ROOT, "paper_1808_00270_gb300", "csrc", "k_history.cu")
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def measured_traffic(workload: str):
    """DRAM bytes per launch of the history convolution from the committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(PROFILES, "hist_conv_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if d.get("kernel_source_sha256_16") != kernel_source_hash() or d.get("workload") != workload:
        return None
    return d.get("dram_bytes_per_launch")


def peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def run_oracle(w, pos, vel, ks, g, f, dr, steps: int, seconds: float):
    """The FP64 oracle as it stands on the host cores: one untimed step, then
    full steps until `steps` or the time budget is reached."""
    import oracle
    s = oracle.System(n=w.n, box=w.box, mass=w.mass, kT=w.kT, dt=w.dt, m_max=w.m_max, r_c=w.r_c,
                      A_cons=w.A_cons, seed=w.seed, pos=pos, vel=vel)
    assert s.set_kernels(ks, g=g, f=f, dr=dr) == 0
    s.step(1)
    done, t0 = 0, time.perf_counter()
    while done < steps:
        s.step(1)
        done += 1
        if time.perf_counter() - t0 > seconds:
            break
    el = time.perf_counter() - t0
    return w.n * done / el, done, el, oracle.threads()


def main():
    args = parse()
    rank, world, local = dist_env()
    from paper_1808_00270_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    ks = inputs.self_kernel_samples(w)
    g, f, dr = inputs.pair_kernel_tables(w)
    cfg = dict(w.describe())
    cfg.update({"global_batch": w.n * world, "parallelism": f"replicas{world}",
                "l2": "inputs larger than L2: 1.26 GB FP32 history ring streamed every step"})

    if args.impl == "reference":
        if rank != 0:
            return 0
        pos, vel = inputs.initial_state(w)
        val, done, el, cores = run_oracle(w, pos, vel, ks, g, f, dr, args.steps, args.reference_seconds)
        sample = (f"{done} full FP64 oracle steps of the {w.n}-particle, m_max={w.m_max} workload after one "
                  f"untimed step ({el:.1f} s); {args.steps} steps requested")
        print(json.dumps({"metric": METRIC, "value": val, "unit": UNIT, "impl": "reference", "n_gpus": 0,
                          "steps": done, "warmup": 1, "ms_per_step": 1e3 * el / max(done, 1),
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": cfg,
                          "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                                           "sample": sample},
                          "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return 0

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    init_replicas(world, local, "nccl")
    from paper_1808_00270_gb300 import GLD, build as gbuild
    gbuild.build()

    pos, vel = inputs.initial_state(w, seed=w.seed + rank)
    vacf = dict(vacf_len=w.m_max, vacf_stride=max(1, w.m_max // 10), vacf_burnin=2 * w.m_max)
    common = dict(n=w.n, box=w.box, mass=w.mass, kT=w.kT, dt=w.dt, m_max=w.m_max, r_c=w.r_c, A_cons=w.A_cons,
                  seed=w.seed + rank, hist_dtype=args.hist, kahan=args.kahan, **vacf)
    sim = GLD(pos=pos, vel=vel, **common)
    sim.set_kernels(ks, g=g, f=f, dr=dr)
    T = 64
    # warm-up: at least W steps, then up to a noise-block boundary and one graph replay
    sim.step(max(args.warmup, 3))
    sim.step((-sim.step_index) % T + T)
    sim.sync()

    K = args.steps
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] if os.environ.get("CUDA_VISIBLE_DEVICES") else str(local)
    os.makedirs(os.path.join(ROOT, "gpurun_out"), exist_ok=True)
    clocks = ClockSampler(gpu_index, os.path.join(ROOT, "gpurun_out", f"clocks_rank{rank}.csv"))
    time.sleep(0.5)
    stream = torch.cuda.current_stream()
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sim.step(K)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    sim.sync()
    ms = max_over_ranks(ms, world, "cuda")
    value = replica_value(w.n, K, world, ms)
    blocks = (K + T - 1) // T
    launches = K * (7 if w.m_max > 0 else 6) + 2 * blocks

    # per-kernel device time with CUDA events on the same stream
    prof = sim.profile_steps(args.profile_steps)
    h_ms, h_n = prof["hist_conv"]
    nacc = 2
    alg_bytes = (4 * 3 * (w.m_max - 1) + 4 * 3 * nacc) * w.n * (0.5 if args.hist == "bf16" else 1.0)
    if args.hist == "bf16":
        alg_bytes = (2 * 3 * (w.m_max - 1) + 4 * 3 * nacc) * w.n
    avg_s = h_ms / 1e3 / max(h_n, 1)
    achieved = alg_bytes / avg_s / 1e9
    peak, peak_kind = peaks()
    total_ms = sum(v[0] for v in prof.values())
    roofline = {"bound": "hbm", "kernel": "hist_conv", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
                "traffic": measured_traffic(args.workload), "algorithmic_bytes_per_launch": alg_bytes,
                "avg_launch_ms": avg_s * 1e3,
                "kernel_share": {k: v[0] / total_ms for k, v in prof.items() if total_ms > 0}}

    diag = sim.diag()
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e = GLD(pos=pos, vel=vel, **common)
        e.set_kernels(ks, g=g, f=f, dr=dr)
        e.step(K)
        cv, _ = e.vacf()
        p_out, v_out = e.get_state()
        t1 = time.perf_counter()
        e.close()
        h2d = 2 * 16 * w.n + 8 * (1 + 2) * w.m_max + 4 * f.size
        d2h = 2 * 16 * w.n + 16 * w.m_max + 8
        e2e = {"value": w.n * K / (t1 - t0), "unit": UNIT, "h2d_bytes_per_step": h2d / K,
               "d2h_bytes_per_step": d2h / K,
               "what": "gld_create from host arrays + gld_set_kernels + gld_step(K) + gld_vacf + gld_get_state"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        val, done, el, cores = run_oracle(w, pos, vel, ks, g, f, dr, 1000, 20.0)
        cpu = {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{done} full FP64 oracle steps of the same {w.n}-particle workload after one untimed "
                         f"step ({el:.1f} s)"}

    if rank == 0:
        print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                          "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "bf16-history" if args.hist == "bf16" else "f32",
                          "data": "synthetic", "config": cfg, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                          "clocks": clk, "gpu_launches": launches, "diag": diag, "profile": {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items()}}))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
