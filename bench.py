"""Benchmark of the fused collide-and-stream step (MLUPS and HBM roofline).

Default workload: the 256x1024 channel sweep -- nine simulations, Gibbs
elasticity beta in {0.05, 0.1, 0.2} x quadratic sensitivity sigma_TT in
{5e-4, 1e-3, 2e-3}, bubble R=32 a quarter of the way along the channel,
density ratio 10, FP32 storage.  One benchmark step advances every
simulation of the batch by one time step: by default one launch of the
batched streaming step kernel over all nine (--mode plain: nine launches,
one per simulation).  Each simulation's 75 MB state has been evicted from the 129 MB
L2 by the other eight before it is read again.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs its own copy of the batch (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
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

import numpy as np  # noqa: E402

import seeded_inputs as si  # noqa: E402

# algorithmic bytes per fluid node and step: read + write of the node's
# state -- 36 FP32 populations; or, with 16-bit storage, 36 16-bit deviations
# and the float4 of rest-state moments
BYTES_PER_NODE_STEP = {"fp32": 288, "fp16": 176, "bf16": 176}
BYTES_PER_NODE_BUFFER = {"fp32": 144, "fp16": 88, "bf16": 88}
PRECISION_CODE = {"fp32": 0, "fp16": 1, "bf16": 2}
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
KERNEL_SRC = os.path.join(ROOT, "paper_2408_00146_gb300", "csrc", "lbm_kernels.cu")


def workload(name: str) -> list[dict]:
    if name == "channel_256x1024_sweep":
        return si.channel_256x1024_sweep()
    if name == "channel_1024x4096":
        return [si.channel_1024x4096()]
    if name == "channel_64x128":
        return [si.channel_64x128()]
    if name == "ensemble_64":
        # 64 channels of uneven size (nx 128..512, ny = 4 nx) and physics
        return si.ensemble_channels(64, seed=0)
    if name == "channel_512x1024":
        # profiling case: one lattice with 150 MB of populations (> L2)
        p = si.channel_256x1024()
        p.update(nx=512, xb=256.0)
        return [p]
    raise SystemExit(f"unknown workload {name}")


def fluid_nodes(p: dict) -> int:
    return p["nx"] * (p["ny"] - 2 if p["walls"] else p["ny"])


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def kernel_hash() -> str:
    with open(KERNEL_SRC, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def streams(p: dict) -> bool:
    """Whether the library steps this FP32 lattice with the y-streaming
    kernel (walls, nx a multiple of 32, at least 16 fluid rows)."""
    return bool(p["walls"]) and p["nx"] % 32 == 0 and p["ny"] - 2 >= 16


def step_kernel_name(mode: str, precision: str, params=None) -> str:
    if precision == "fp32":
        if params and all(streams(p) for p in params):
            return "stream_batch_kernel"
        return "step_batch_kernel" if mode == "batched" else "step_kernel"
    return "step_batch_dev_kernel" if mode == "batched" else "step_dev_kernel"


def profiled_traffic(work: str, mode: str, precision: str, params=None):
    """DRAM bytes per step-kernel launch from the committed ncu summary, if it
    was taken on the current kernel source for this workload and launch."""
    if not os.path.exists(PROFILE_TRAFFIC):
        return None
    with open(PROFILE_TRAFFIC) as fh:
        d = json.load(fh)
    ent = d.get(f"{work}/{precision}/{step_kernel_name(mode, precision, params)}")
    if not ent or ent.get("kernel_sha256_16") != kernel_hash():
        return None
    return float(ent["dram_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def max_over_ranks(ms: float, device: str) -> float:
    """Maximum of a per-rank time over all ranks (identity without a process
    group).  The only collective of the benchmark: the simulations are
    independent, nothing on the data path is exchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(ms_max: float, nodes_per_step: int, steps: int, world: int) -> float:
    """Whole-job MLUPS: every rank advanced its own copy of the batch."""
    return nodes_per_step * steps * world / (ms_max * 1e-3) / 1e6


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- CPU oracle
def oracle_rate(params: dict, steps: int, threads: int) -> tuple[float, int, float]:
    """MLUPS of the FP64 CPU oracle over `steps` steps of `params`."""
    from oracle import oracle as orc
    used = orc.set_threads(threads)
    o = orc.Oracle(params)
    o.init_fields(si.bubble_fields(params))
    o.step(1)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    o.close()
    return fluid_nodes(params) * steps / dt / 1e6, used, dt


def cpu_baseline(work: str, budget_s: float = 15.0) -> dict:
    params = workload(work)[0]
    threads = os.cpu_count() or 1
    rate1, used, dt1 = oracle_rate(params, 1, threads)
    steps = max(1, min(1000, int(budget_s / max(dt1, 1e-6))))
    rate, used, dt = oracle_rate(params, steps, threads)
    # the same oracle on one core, for a few seconds
    rate_1, _, dt_1 = oracle_rate(params, max(1, steps // max(used, 1) // 3), 1)
    return {"value": rate, "unit": "MLUPS", "cores": used, "kind": "oracle",
            "sample": f"{steps} FP64 time steps of the first lattice of the workload "
                      f"({params['nx']}x{params['ny']}), {dt:.1f} s",
            "single_core_value": rate_1}


def run_reference(args) -> None:
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    work = workload(args.workload)
    # each benchmark step is a bounded sample: one FP64 oracle time step of a
    # 64x128 channel with the physics of the next member of the workload
    from oracle import oracle as orc
    threads = os.cpu_count() or 1
    used = orc.set_threads(threads)
    sims = []
    for p in work:
        q = dict(p)
        q.update(nx=64, ny=128, R=12.0, xb=32.0, yb=40.0)
        o = orc.Oracle(q)
        o.init_fields(si.bubble_fields(q))
        sims.append((q, o))
    for k in range(args.warmup):
        sims[k % len(sims)][1].step(1)
    t0 = time.perf_counter()
    nodes = 0
    for k in range(args.steps):
        q, o = sims[k % len(sims)]
        o.step(1)
        nodes += fluid_nodes(q)
    dt = time.perf_counter() - t0
    v = nodes / dt / 1e6
    print(json.dumps({
        "impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / max(args.steps, 1) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample": "one oracle step of a 64x128 "
                   "channel per benchmark step, physics of the workload members"},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": used, "kind": "oracle",
                         "sample": "64x128 channel, one FP64 step per benchmark step"},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------- GPU arm
def run_gpu(args) -> None:
    import torch
    import torch.distributed as dist

    from paper_2408_00146_gb300 import lbm

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev_index = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    params = workload(args.workload)
    for p in params:
        p["precision"] = PRECISION_CODE[args.precision]
    nodes_per_step = sum(fluid_nodes(p) for p in params)

    sims = [lbm.Sim(p, stream=stream, workspace="torch") for p in params]
    for s in sims:
        s.init()                      # analytic initial state, built on the device
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def step_all():
        if args.mode == "batched":
            lbm.lbm_step_batch(sims, 1)       # one launch over every simulation
        else:
            for s in sims:                   # one launch per simulation
                s.step(1)

    def timed(nsteps):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        l0 = sum(s.launches() for s in sims)
        ev0.record(stream)
        if args.mode == "batched" and not args.per_step_calls:
            lbm.lbm_step_batch(sims, nsteps)  # one call: replayed CUDA graphs of 64 steps
        elif args.graph and args.mode == "plain":
            for s in sims:                   # all steps in one call: CUDA-graph replay
                s.step(nsteps)
        else:
            for _ in range(nsteps):
                step_all()
        ev1.record(stream)
        barrier()
        return ev0.elapsed_time(ev1), sum(s.launches() for s in sims) - l0

    # measured strip plan of the batched launch (steps outside the timed region)
    tuned_steps = 0
    if args.mode == "batched" and args.tune_steps > 0:
        tuned_steps = lbm.lbm_tune_batch(sims, args.tune_steps)
    plan = lbm.lbm_batch_plan(sims)
    warmup_run = args.warmup
    if args.mode == "batched" and not args.per_step_calls:
        # at least one 64-step run, so that the batch's graph is captured
        # before the timed region
        warmup_run = max(args.warmup, 64)
        lbm.lbm_step_batch(sims, warmup_run)
    else:
        for _ in range(args.warmup):
            step_all()
    with ClockSampler(dev_index) as clk:
        ms, launches = timed(args.steps)
    clocks = clk.summary()

    ms_max = max_over_ranks(ms, "cuda")
    value = weak_scaling_value(ms_max, nodes_per_step, args.steps, ws)

    # roofline of the dominant kernel: every launch in the timed region is the
    # fused step kernel (one simulation, or the whole batch, per launch)
    per_launch_ms = ms / launches
    sims_per_launch = len(params) if args.mode == "batched" else 1
    bpn = BYTES_PER_NODE_STEP[args.precision]
    per_launch_bytes = bpn * nodes_per_step / len(params) * sims_per_launch
    peaks = measured_peaks()
    achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
    kernel = step_kernel_name(args.mode, args.precision, params)
    traffic = profiled_traffic(args.workload, args.mode, args.precision, params)

    # the other launch mode on the same simulations, for comparison
    other = None
    if args.compare_modes and len(params) > 1:
        mode = args.mode
        args.mode = "plain" if mode == "batched" else "batched"
        ms_o, _ = timed(max(args.steps // 4, 1))
        other = {"mode": args.mode,
                 "value": nodes_per_step * max(args.steps // 4, 1) / (ms_o * 1e-3) / 1e6}
        args.mode = mode

    e2e = run_e2e(args, lbm, torch, stream, params) if not args.no_e2e else None
    served = run_served(args, torch) if (args.serve_requests > 0 and rank == 0) else None

    for s in sims:
        s.close()
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload)
    if rank == 0:
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "lattices": [f"{p['nx']}x{p['ny']}" for p in params],
                       "sims_per_gpu": len(params), "fluid_nodes_per_step": nodes_per_step,
                       "launch_mode": args.mode + (" graph" if (args.graph and args.mode == "plain") or
                                                   (args.mode == "batched" and not args.per_step_calls)
                                                   else ""),
                       "warmup_steps_run": warmup_run,
                       "other_mode": other,
                       "strip_plan": {"tuned": tuned_steps > 0, "tuning_steps": tuned_steps,
                                      "strip_chunks": sorted(set(plan) - {0})},
                       "storage": args.precision,
                       "l2": "working set %.0f MB > 129 MB L2; simulations interleaved per step"
                             % (sum(2 * BYTES_PER_NODE_BUFFER[args.precision] * p["nx"] * p["ny"]
                                    for p in params) / 1e6),
                       "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                         "traffic": traffic, "peak_source": peaks["source"],
                         "kernel": kernel, "bytes_per_node_step": bpn},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "served": served,
            "gpu_launches": launches,
            "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                       "reasons": clocks["reasons"]},
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_served(args, torch) -> dict:
    """The served workload: a Poisson stream of requests (uneven lattices,
    physics and storage precisions) through the serving loop, arrivals in
    wall time; p50/p99 of arrival-to-finish latency and aggregate MLUPS."""
    from paper_2408_00146_gb300.serve import LbmEngine, Server, requests_from_stream, summary

    stream = si.request_stream(n=args.serve_requests, rate=args.serve_rate, seed=0)
    reqs = requests_from_stream(stream, max_steps=args.serve_max_steps, tol=1e-6)
    free, _total = torch.cuda.mem_get_info()
    budget = int(min(150e9, 0.8 * free))
    srv = Server(LbmEngine(), budget_bytes=budget, round_steps=100)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = srv.run(reqs)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    out = summary(res, wall, srv.node_steps)
    out.update({"rate_per_s": args.serve_rate, "max_steps": args.serve_max_steps,
                "tol": 1e-6, "round_steps": 100, "budget_gb": budget / 1e9,
                "peak_resident": srv.peak_resident, "peak_gb": srv.peak_bytes / 1e9,
                "fp16_requests": sum(p["precision"] == 1 for _, p in stream),
                "lattices": "nx log-uniform 64..512 (x16), ny = 4 nx"})
    return out


def run_e2e(args, lbm, torch, stream, params) -> dict:
    """Same metric through the public C ABI with host buffers: initial fields
    from the host, steps, the observables read back every 100 steps and the
    final fields copied to the host, all inside the timed region."""
    steps = max(args.e2e_steps, 1)
    host_in = [si.bubble_fields(p) for p in params]   # params carry the precision
    host_out = [np.empty((6, p["ny"], p["nx"])) for p in params]
    sims = [lbm.Sim(p, stream=stream, workspace="torch") for p in params]
    torch.cuda.synchronize()
    h2d = d2h = 0
    t0 = time.perf_counter()
    for s, f in zip(sims, host_in):
        s.init(f)
        h2d += f.size * 4                       # fields cross as FP32
    done = 0
    while done < steps:
        n = min(100, steps - done)
        if args.mode == "batched":
            lbm.lbm_step_batch(sims, n)   # as in the device-timed loop
        else:
            for _ in range(n):            # interleaved, as in the device-timed loop
                for s in sims:
                    s.step(1)
        for s in sims:
            s.observe()
            d2h += 8 * 8
        done += n
    for s, out in zip(sims, host_out):
        lbm.lbm_observe(s.handle, out)
        d2h += out.size * 4 + 8 * 8
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    for s in sims:
        s.close()
    nodes = sum(fluid_nodes(p) for p in params) * steps
    return {"value": nodes / dt / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "steps": steps}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="channel_256x1024_sweep",
                    choices=["channel_256x1024_sweep", "channel_1024x4096", "channel_64x128",
                             "channel_512x1024", "ensemble_64"])
    ap.add_argument("--mode", default="batched", choices=["batched", "plain"],
                    help="batched: one launch per step over all simulations; "
                         "plain: one launch per simulation")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16"],
                    help="population storage (arithmetic is FP32 in every case)")
    ap.add_argument("--graph", action="store_true",
                    help="plain mode: advance each simulation by all timed steps in one "
                         "lbm_step call (replayed CUDA graphs of 64 steps)")
    ap.add_argument("--per-step-calls", action="store_true",
                    help="batched mode: one lbm_step_batch call per step instead of one call for "
                         "all timed steps (no CUDA-graph replay)")
    ap.add_argument("--compare-modes", action="store_true", default=True)
    ap.add_argument("--tune-steps", type=int, default=10,
                    help="batched mode: steps per candidate strip plan for lbm_tune_batch "
                         "before the warm-up (0: the cost model's plan)")
    ap.add_argument("--e2e-steps", type=int, default=1000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=48,
                    help="requests of the served workload (0: skip it)")
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-max-steps", type=int, default=3000)
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
