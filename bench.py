#!/usr/bin/env python
"""GLD throughput on one GB300: particle-steps/s of the 262144-particle,
m_max = 400 suspension (FP32 history ring of 1.26 GB, larger than L2).

One step = the whole hot path: history convolution, pair dissipative force
and position update, cell-list rebuild, conservative force and velocity
update, VACF accumulation, and the colored-noise block every 64 steps.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead.
Under torchrun each rank steps an independent replica (different seed); there
is no data-path collective, only a barrier and a max over ranks of the time.

The headline line also summarises the first requests of the serving trace
(`served`).  Two more workloads print their own line:
  --workload batch512  512 uneven independent systems stepped as one batch,
                       against the same systems stepped one at a time;
  --workload serve     the seeded 1000-request Poisson trace (50/s) served
                       with continuous batching, against the same requests
                       run one at a time (`--requests R` keeps the first R).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
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
    ap.add_argument("--serve-requests", type=int, default=60,
                    help="requests of the serving trace summarised in the headline line (0: none)")
    ap.add_argument("--graph-form", default="conditional", choices=["conditional", "gated"],
                    help="gated: rebuild kernels gated on the device instead of a conditional graph node "
                         "(every graph node a plain kernel, which per-kernel profilers can capture)")
    ap.add_argument("--modes", action="store_true",
                    help="memory sums in auxiliary-variable form (the workload's kernels are sums of damped modes) "
                         "instead of the history-ring convolution")
    ap.add_argument("--pcorr", type=int, default=0,
                    help="also accumulate the distance-binned pair correlations on this many bins of [0, r_c)")
    ap.add_argument("--pair-noise", type=int, default=0,
                    help="pair-correlated random force with a Chebyshev form of this degree on an interval of the "
                         "pair matrix's spectrum (estimated by a Lanczos run, checked at every noise block); the "
                         "workload's full-strength pair kernel")
    ap.add_argument("--pair-noise-lanczos", type=int, default=-1, choices=[-1, 0, 1],
                    help="pair-correlated random force by Algorithm 1 (a Lanczos iteration per frequency, tol 1e-6, "
                         "at most 24 vectors; eager steps): 0 every step, 1 one run per 64-step block over the time "
                         "window; the workload's full-strength pair kernel")
    ap.add_argument("--skin", type=float, default=0.0,
                    help="Verlet-list skin (0: the library's choice); results do not depend on it")
    ap.add_argument("--hist", default="f32", choices=["f32", "bf16"])
    ap.add_argument("--kahan", action="store_true")
    ap.add_argument("--reference-seconds", type=float, default=120.0)
    ap.add_argument("--systems", type=int, default=512, help="batch512: number of systems")
    ap.add_argument("--requests", type=int, default=1000, help="serve: requests of the trace (its first R)")
    ap.add_argument("--max-members", type=int, default=0, help="serve: systems stepped together at most")
    ap.add_argument("--hbm-budget", type=float, default=0.0, help="serve: device GB for admitted systems")
    ap.add_argument("--sequential", type=int, default=-1,
                    help="serve: requests also run one at a time with plain gld_step (-1: all)")
    ap.add_argument("--batch-systems", type=int, default=512,
                    help="systems of the batched workload summarised in the headline line (0: none)")
    ap.add_argument("--clock-log", default=None,
                    help="file for the nvidia-smi clock samples of the timed region (default: a temporary file)")
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
    """nvidia-smi samples of SM clock and throttle reasons during the timed
    region (a read-only query), kept in a temporary file or in `path`."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str, path: str | None = None):
        self.proc, self.tmp = None, path is None
        if path is None:
            fd, path = tempfile.mkstemp(prefix="gld_clocks_", suffix=".csv")
            os.close(fd)
        self.path = path
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
        if self.tmp:
            os.remove(self.path)
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


def pctl(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs, dtype=float), q)) if len(xs) else None


def batch_leg(args, rank: int, world: int, local: int, quiet: bool = False):
    """Independent uneven systems stepped as one batch (one launch per kernel
    family per step, 64-step blocks as one graph) against the same systems
    stepped one at a time with plain gld_step."""
    import numpy as np
    import torch
    from paper_1808_00270_gb300 import GLD, Batch, inputs
    torch.cuda.set_device(local)
    ws = inputs.batch_systems(args.systems, seed=4 + 1000 * rank)
    vacf = dict(vacf_len=100, vacf_stride=10)
    systems = []
    for w in ws:
        pos, vel = inputs.initial_state(w)
        g = GLD(pos=pos, vel=vel, n=w.n, box=w.box, mass=w.mass, kT=w.kT, dt=w.dt, m_max=w.m_max, r_c=w.r_c,
                A_cons=w.A_cons, seed=w.seed, hist_dtype=args.hist, kahan=args.kahan, **vacf)
        gk, f, dr = inputs.pair_kernel_tables(w)
        g.set_kernels(inputs.self_kernel_samples(w), g=gk, f=f, dr=dr)
        systems.append(g)
    n_tot = sum(w.n for w in ws)
    b = Batch()
    for g in systems:
        b.add(g)
    T = 64
    K = max(T, (args.steps + T - 1) // T * T)
    b.step(T * max(1, (args.warmup + T - 1) // T))  # schedule timing, graph capture
    b.sync()
    stream = torch.cuda.current_stream()
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]
    clocks = ClockSampler(gpu_index, args.clock_log)
    time.sleep(0.5)
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    b.step(K)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    b.sync()
    ms = max_over_ranks(ms, world, "cuda")
    value = world * n_tot * K / (ms / 1e3)
    info = b.info()
    for g in systems:  # members stay usable alone
        b.remove(g)
    # the same systems one at a time (each replays its own captured 64-step graph)
    for g in systems:
        g.step(T)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for g in systems:
        g.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    seq = world * n_tot * K / (ms_seq / 1e3)
    elem = 2 if args.hist == "bf16" else 4
    alg = sum((elem * 3 * (w.m_max - 1) + 4 * 3 * 2) * w.n for w in ws)
    conv_ms = info["schedule_ms"][info["schedule"]]
    peak, peak_kind = peaks()
    hist_bytes = sum(elem * 3 * (w.m_max - 1) * ((w.n + 31) // 32 * 32) for w in ws)
    out = {"metric": f"GLD particle-steps/s, {len(ws)} batched uneven systems", "value": value,
           "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": ms / K,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16-history" + ("+kahan" if args.kahan else "") if args.hist == "bf16" else
           ("f32+kahan" if args.kahan else "f32"), "data": "synthetic",
           "config": {"workload": f"batch{len(ws)}", "systems": len(ws), "particles": n_tot,
                      "n_range": [min(w.n for w in ws), max(w.n for w in ws)],
                      "m_max_set": sorted({w.m_max for w in ws}), "history_bytes": hist_bytes,
                      "parallelism": f"replicas{world}",
                      "l2": f"inputs larger than L2: {hist_bytes / 1e9:.2f} GB of history rings streamed every step"},
           "sequential": {"value": seq, "unit": UNIT, "ms_per_step": ms_seq / K,
                          "what": "the same systems one after another, each gld_step(K) replaying its own graph"},
           "speedup_vs_sequential": value / seq,
           "autotune": {"schedule": info["schedule"], "schedule_ms": info["schedule_ms"],
                        "schedules": ["256-column tiles, longest memory first", "128-column tiles, longest first",
                                      "256-column tiles, member order", "one block per system"]},
           "roofline": {"bound": "hbm", "kernel": "b_conv (batched history convolution)",
                        "achieved": alg / (conv_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": alg / (conv_ms / 1e3) / 1e9 / peak, "peak_source": f"{peak_kind} hbm_gbs",
                        "traffic": None, "algorithmic_bytes_per_launch": alg, "avg_launch_ms": conv_ms},
           "clocks": clk, "gpu_launches": (K // T) * (2 + T * 8)}
    if rank == 0 and not quiet:
        print(json.dumps(out))
    for g in systems:
        g.close()
    b.close()
    return out


def request_inputs(trace, vacf):
    """Host inputs of each request of a trace (drawn before the clock starts)."""
    from paper_1808_00270_gb300 import inputs
    out = []
    for r in trace:
        w = r.w
        pos, vel = inputs.initial_state(w)
        gk, f, dr = inputs.pair_kernel_tables(w)
        out.append(dict(n=w.n, box=w.box, dt=w.dt, m_max=w.m_max, r_c=w.r_c, pos=pos, vel=vel,
                        Ks=inputs.self_kernel_samples(w), g=gk, f=f, dr=dr, steps=r.steps, mass=w.mass, kT=w.kT,
                        A_cons=w.A_cons, seed=w.seed, **vacf))
    return out


def serve_requests(srv, trace, reqs, t0):
    return [srv.submit(arrival=t0 + r.arrival, **q) for r, q in zip(trace, reqs)]


def serve_leg(args, rank: int, world: int, local: int, quiet: bool = False):
    """The seeded Poisson trace served with continuous batching, against the
    same requests run one at a time with plain gld_step (FIFO queue)."""
    import numpy as np
    import torch
    from paper_1808_00270_gb300 import GLD, Server, inputs
    torch.cuda.set_device(local)
    trace = inputs.serve_trace(1000, seed=5 + 1000 * rank)[: args.requests]
    vacf = dict(vacf_len=100, vacf_stride=10)
    budget = int(args.hbm_budget * 1e9)
    # warm-up: module load, schedule timing and capture paths on a throw-away server
    warm = Server(hbm_budget=budget, max_members=args.max_members)
    wt = inputs.serve_trace(4, seed=99)
    serve_requests(warm, wt, request_inputs(wt, vacf), 0.0)
    warm.drain(600)
    warm.close()
    reqs = request_inputs(trace, vacf)
    srv = Server(hbm_budget=budget, max_members=args.max_members)
    t_sub = time.perf_counter()
    t0 = srv.clock() + 0.5 + 0.002 * len(trace)  # submission ends before the first arrival
    ids = serve_requests(srv, trace, reqs, t0)
    sub_s = time.perf_counter() - t_sub
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]
    clocks = ClockSampler(gpu_index, args.clock_log)
    srv.drain(3600)
    clk = clocks.stop()
    res = [srv.result(i) for i in ids]
    st = srv.stats()
    ok = [r for r in res if r["status"] == 0]
    lat = [r["done"] - r["arrival"] for r in ok]
    t_end = max(r["done"] for r in ok)
    work = sum(r.w.n * r.steps for r, x in zip(trace, res) if x["status"] == 0)
    t_end = float(t_end)
    served = {"p50_s": pctl(lat, 50), "p99_s": pctl(lat, 99), "mean_s": float(np.mean(lat)),
              "throughput": work / (t_end - t0), "unit": UNIT, "makespan_s": t_end - t0,
              "done": len(ok), "failed": len(res) - len(ok), "blocks": st["blocks"],
              "members_peak": st["members_peak"], "bytes_peak": st["bytes_peak"], "budget": st["budget"],
              "queue_wait_p50_s": pctl([r["admitted"] - r["arrival"] for r in ok], 50)}
    srv.close()
    # sequential plain runs of the same requests, FIFO in arrival order
    nseq = len(trace) if args.sequential < 0 else min(args.sequential, len(trace))
    seq = None
    if nseq > 0:
        svc = []
        for r, q in zip(trace[:nseq], reqs):
            w = r.w
            torch.cuda.synchronize()
            a = time.perf_counter()
            g = GLD(pos=q["pos"], vel=q["vel"], n=w.n, box=w.box, mass=w.mass, kT=w.kT, dt=w.dt, m_max=w.m_max,
                    r_c=w.r_c, A_cons=w.A_cons, seed=w.seed, **vacf)
            g.set_kernels(q["Ks"], g=q["g"], f=q["f"], dr=q["dr"])
            g.step(r.steps)
            g.vacf()
            svc.append(time.perf_counter() - a)
            g.close()
        done_t, lat_s = 0.0, []
        for r, sv in zip(trace[:nseq], svc):
            start = max(r.arrival, done_t)
            done_t = start + sv
            lat_s.append(done_t - r.arrival)
        wseq = sum(r.w.n * r.steps for r in trace[:nseq])
        seq = {"requests": nseq, "p50_s": pctl(lat_s, 50), "p99_s": pctl(lat_s, 99), "throughput": wseq / sum(svc),
               "unit": UNIT, "what": "each request alone: gld_create + gld_set_kernels + gld_step + gld_vacf, "
                                     "FIFO in arrival order (latency from the measured service times)"}
    mean_work = work / max(len(ok), 1)
    out = {"metric": f"GLD served p99 latency ({len(trace)}-request Poisson trace, 50/s)",
           "value": served["p99_s"], "unit": "s", "n_gpus": world, "steps": int(sum(r.steps for r in trace)),
           "warmup": 4, "ms_per_step": None, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"serve{len(trace)}", "requests": len(trace), "rate_per_s": 50.0,
                      "n_range": [512, 65536], "m_max_range": [64, 400], "step_range": [2000, 20000],
                      "density_range": [0.02, 0.2], "vacf": vacf, "max_members": args.max_members,
                      "parallelism": f"replicas{world}", "submission_s": sub_s},
           "served": served, "sequential": seq,
           "throughput_vs_sequential": served["throughput"] / seq["throughput"] if seq else None,
           "max_sustainable_rate_per_s": served["throughput"] / mean_work,
           "clocks": clk, "gpu_launches": st["blocks"] * (2 + 64 * 8)}
    if rank == 0 and not quiet:
        print(json.dumps(out))
    return out


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.workload.startswith("batch") and args.impl == "gld":
        batch_leg(args, rank, world, local)
        return 0
    if args.workload.startswith("serve") and args.impl == "gld":
        serve_leg(args, rank, world, local)
        return 0
    from paper_1808_00270_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    ks = inputs.self_kernel_samples(w)
    g, f, dr = inputs.pair_kernel_tables(w)
    cfg = dict(w.describe())
    if args.pcorr > 0:
        cfg["pair_correlation_bins"] = args.pcorr
    if args.modes:
        cfg["memory"] = "auxiliary-variable modes (O(1) per particle-step in m_max)"
    if args.pair_noise > 0:
        cfg["pair_noise"] = {"degree": args.pair_noise, "pair_kernel_scale": 1.0}
    if args.pair_noise_lanczos >= 0:
        cfg["pair_noise"] = {"lanczos_window": args.pair_noise_lanczos, "tol": 1e-6, "kmax": 24,
                             "pair_kernel_scale": 1.0}
    cfg.update({"global_batch": w.n * world, "parallelism": f"replicas{world}",
                "l2": "inputs larger than L2: 1.26 GB FP32 history ring streamed every step"})
    if args.skin > 0:
        cfg["skin"] = args.skin

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
                  seed=w.seed + rank, hist_dtype=args.hist, kahan=args.kahan,
                  use_graphs=2 if args.graph_form == "gated" else 1, skin=args.skin, **vacf)
    sim = GLD(pos=pos, vel=vel, **common)
    sim.set_kernels(ks, g=g, f=f, dr=dr)
    if args.pcorr > 0:
        sim.set_pair_correlation(args.pcorr, w.r_c)
    if args.modes:
        sim.set_memory_modes(*inputs.memory_modes(w))
    if args.pair_noise > 0:
        # one untimed block first: the synthetic positions start with close
        # contacts that the conservative force removes within a few steps,
        # and the interval is estimated on the relaxed spectrum
        sim.step(64)
        lo, hi, cheb = sim.set_pair_noise_on(args.pair_noise)
        cfg["pair_noise"].update({"interval": [lo, hi], "interpolation_error": cheb,
                                  "interval_estimated_at_step": 64})
    if args.pair_noise_lanczos >= 0:
        sim.set_pair_noise_lanczos(1e-6, 24, window=args.pair_noise_lanczos)
    T = 64
    # warm-up: at least W steps and until the VACF runs with every origin in
    # flight (burn-in + vacf_len steps), so the clock sees its full cost; then
    # up to a noise-block boundary (the timed region starts with a whole
    # block's noise) and one graph replay
    warm = max(args.warmup, 3, vacf["vacf_burnin"] + vacf["vacf_len"])
    sim.step(warm)
    sim.step((-sim.step_index) % T + T)
    sim.sync()
    warm_steps = sim.step_index

    K = args.steps
    d0 = sim.diag()  # before the clock: graph form and list builds so far
    _, orig0 = sim.vacf()
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] if os.environ.get("CUDA_VISIBLE_DEVICES") else str(local)
    clocks = ClockSampler(gpu_index, args.clock_log)
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
    d1 = sim.diag()
    _, orig1 = sim.vacf()
    ms = max_over_ranks(ms, world, "cuda")
    value = replica_value(w.n, K, world, ms)
    blocks = (K + T - 1) // T

    # per-kernel device time with CUDA events on the same stream (the Lanczos
    # forms decide on the host between launches: profiled without them)
    if args.pair_noise_lanczos >= 0:
        kdim = sim.diag()["krylov_iterations"]
        sim.set_pair_noise_lanczos(0.0)
        cfg["pair_noise"]["krylov_dimension"] = kdim
        cfg["pair_noise"]["kernel_profile"] = "without the pair noise"
    prof = sim.profile_steps(args.profile_steps)
    h_ms, h_n = prof["hist_conv"]
    nacc = 2
    alg_bytes = (4 * 3 * (w.m_max - 1) + 4 * 3 * nacc) * w.n * (0.5 if args.hist == "bf16" else 1.0)
    if args.hist == "bf16":
        alg_bytes = (2 * 3 * (w.m_max - 1) + 4 * 3 * nacc) * w.n
    kname, traffic = "hist_conv", measured_traffic(args.workload)
    if args.modes:  # per column: Y' of every mode read and written, two ring values, the projections
        nm = len(inputs.memory_modes(w)[0])
        elem = 2 if args.hist == "bf16" else 4
        alg_bytes = 3 * ((w.n + 31) // 32 * 32) * (16 * nm + 2 * elem + 4 * nacc)
        kname, traffic = "modes_step", None
    avg_s = h_ms / 1e3 / max(h_n, 1)
    achieved = alg_bytes / avg_s / 1e9
    peak, peak_kind = peaks()
    total_ms = sum(v[0] for v in prof.values())
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
                "traffic": traffic, "algorithmic_bytes_per_launch": alg_bytes,
                "avg_launch_ms": avg_s * 1e3,
                "kernel_share": {k: v[0] / total_ms for k, v in prof.items() if total_ms > 0}}

    diag = sim.diag()
    diag.update({"untimed_steps_before_clock": warm_steps, "vacf_origins_before": int(orig0),
                 "vacf_origins_after": int(orig1), "vacf_origins_in_flight": (vacf["vacf_len"] + vacf["vacf_stride"] - 1)
                 // vacf["vacf_stride"]})
    T_blocks = (K + T - 1) // T
    # per step: convolution, pair kernel, F^C with the VACF terms, and the
    # rebuild decision (conditional form) or the four gated rebuild kernels
    if d0["graph_mode"] == 2:  # rebuild kernels only on the steps that rebuild
        launches = K * 4 + 4 * (d1["rebuilds"] - d0["rebuilds"]) + 2 * T_blocks
    else:
        launches = K * 7 + 2 * T_blocks
    if args.pcorr > 0:
        launches += K
    if args.pair_noise > 0:  # Clenshaw sweeps per step; filters and the Lanczos check per block
        launches += args.pair_noise * (K + T_blocks) + (2 + 2 * 32) * T_blocks
    if args.pair_noise_lanczos >= 0:  # eager steps; per run: transform, norm, 4 launches per iteration, output
        iters = 4 * ((cfg["pair_noise"]["krylov_dimension"] + 3) // 4)
        runs = T_blocks if args.pair_noise_lanczos == 1 else K
        launches = K * 7 + 2 * T_blocks + runs * (3 + 4 * iters + (2 if args.pair_noise_lanczos == 1 else 1))
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e = GLD(pos=pos, vel=vel, **common)
        e.set_kernels(ks, g=g, f=f, dr=dr)
        if args.pcorr > 0:
            e.set_pair_correlation(args.pcorr, w.r_c)
        if args.modes:
            e.set_memory_modes(*inputs.memory_modes(w))
        e2e_pn = None
        if args.pair_noise > 0:  # here on the unrelaxed start: a wider interval
            e2e_pn = e.set_pair_noise_on(args.pair_noise)
        if args.pair_noise_lanczos >= 0:
            e.set_pair_noise_lanczos(1e-6, 24, window=args.pair_noise_lanczos)
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
        if e2e_pn is not None:
            e2e["pair_noise"] = {"interval": list(e2e_pn[:2]), "interpolation_error": e2e_pn[2],
                                 "interval_estimated_at_step": 0}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        val, done, el, cores = run_oracle(w, pos, vel, ks, g, f, dr, 1000, 20.0)
        cpu = {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{done} full FP64 oracle steps of the same {w.n}-particle workload after one untimed "
                         f"step ({el:.1f} s)"}

    served = None
    if rank == 0 and world == 1 and args.serve_requests > 0:
        sargs = argparse.Namespace(**vars(args))
        sargs.requests, sargs.sequential = args.serve_requests, args.serve_requests
        sargs.max_members, sargs.hbm_budget = 0, 0.0
        o = serve_leg(sargs, rank, world, local, quiet=True)
        served = {"requests": o["config"]["requests"],
                  "trace": "first requests of the seeded 1000-request Poisson trace (50/s; N 512-65536, "
                           "m_max 64-400, 2000-20000 steps, VACF returned)",
                  "p50_s": o["served"]["p50_s"], "p99_s": o["served"]["p99_s"],
                  "throughput": o["served"]["throughput"], "unit": UNIT,
                  "sequential_p50_s": o["sequential"]["p50_s"], "sequential_p99_s": o["sequential"]["p99_s"],
                  "sequential_throughput": o["sequential"]["throughput"],
                  "throughput_vs_sequential": o["throughput_vs_sequential"],
                  "max_sustainable_rate_per_s": o["max_sustainable_rate_per_s"], "gpu_launches": o["gpu_launches"]}

    batched = None
    if rank == 0 and world == 1 and args.batch_systems > 0:
        bargs = argparse.Namespace(**vars(args))
        bargs.systems, bargs.steps, bargs.warmup = args.batch_systems, 128, 64
        o = batch_leg(bargs, rank, world, local, quiet=True)
        batched = {"systems": o["config"]["systems"], "particles": o["config"]["particles"],
                   "workload": "uneven independent systems (N log-uniform 256-16384, densities 0.02-0.2, "
                               "m_max in {100, 200, 400}) stepped as one batch",
                   "value": o["value"], "unit": UNIT, "ms_per_step": o["ms_per_step"], "steps": o["steps"],
                   "sequential_value": o["sequential"]["value"], "speedup_vs_sequential": o["speedup_vs_sequential"],
                   "autotuned_schedule": o["autotune"]["schedules"][o["autotune"]["schedule"]],
                   "conv_roofline_frac": o["roofline"]["frac"], "gpu_launches": o["gpu_launches"]}

    if rank == 0:
        print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                          "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "bf16-history" if args.hist == "bf16" else "f32",
                          "data": "synthetic", "config": cfg, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                          "clocks": clk, "gpu_launches": launches, "served": served, "batched": batched, "diag": diag, "profile": {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items()}}))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
