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
KERNEL_SRC = [os.path.join(ROOT, "paper_2408_00146_gb300", "csrc", f)
              for f in ("lbm_stream.cu", "lbm_stream_body.cuh", "lbm_device.cuh")]


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
    """Hash of the streaming kernels' sources (dispatch, body, device helpers)."""
    h = hashlib.sha256()
    for path in KERNEL_SRC:
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def streams(p: dict, precision: str) -> bool:
    """Whether the library steps this lattice with a y-streaming kernel:
    nx >= 32 and a multiple of 4 (FP32) or 8 (16-bit storage), at least 16 fluid rows,
    walls or a periodic y axis of whole 8-row chunks."""
    nfy = p["ny"] - 2 if p["walls"] else p["ny"]
    if p["nx"] % (4 if precision == "fp32" else 8) or p["nx"] < 32 or nfy < 16:
        return False
    return bool(p["walls"]) or nfy % 8 == 0


def step_kernel_name(mode: str, precision: str, params=None) -> str:
    if params and all(streams(p, precision) for p in params):
        return "stream32_kernel" if precision == "fp32" else "stream16_kernel"
    if precision == "fp32":
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


class _Nvml:
    """Read-only NVML queries through ctypes (the driver's libnvidia-ml):
    current and maximum SM clock and the active clock-event reasons."""

    CLOCK_SM = 1
    # clock-event reason bits of the NVML API
    REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown",
               0x20: "sw_thermal_slowdown", 0x4: "sw_power_cap"}

    def __init__(self, device_index: int):
        import ctypes
        self.c = ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.lib = lib
        self.h = ctypes.c_void_p()
        uuid = None
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
        except Exception:
            uuid = None
        rc = 1
        if uuid:
            rc = lib.nvmlDeviceGetHandleByUUID(("GPU-" + uuid).encode(), ctypes.byref(self.h))
        if rc != 0:
            rc = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(device_index),
                                                   ctypes.byref(self.h))
        if rc != 0:
            lib.nvmlShutdown()
            raise OSError("no NVML handle for the device")
        self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")

    def sample(self) -> tuple[float, float, list[str]]:
        c = self.c
        sm, mx, rs = c.c_uint(), c.c_uint(), c.c_ulonglong()
        self.lib.nvmlDeviceGetClockInfo(self.h, self.CLOCK_SM, c.byref(sm))
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.CLOCK_SM, c.byref(mx))
        self.reasons_fn(self.h, c.byref(rs))
        return float(sm.value), float(mx.value), [n for b, n in self.REASONS.items()
                                                  if rs.value & b]

    def close(self):
        self.lib.nvmlShutdown()


class ClockSampler:
    """SM clock and throttle samples during the timed region: NVML polled
    from a host thread every 0.2 ms (a region of a few milliseconds still
    gets samples), else nvidia-smi every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.tmp = None
        self.rows: list[tuple[float, float, list[str]]] = []   # inside the region
        self.edges: list[tuple[float, float, list[str]]] = []  # just before and after
        self.source = "nvml"
        self.thread = None
        self.stop = False
        try:
            self.nvml = _Nvml(device_index)
        except (OSError, AttributeError):
            self.nvml = None
            self.source = "nvidia-smi"

    def _poll(self):
        while not self.stop:
            self.rows.append(self.nvml.sample())
            time.sleep(0.0002)

    def __enter__(self):
        if self.nvml is not None:
            import threading
            self.edges.append(self.nvml.sample())
            self.switch = sys.getswitchinterval()
            sys.setswitchinterval(0.0002)
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            return self
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.thread is not None:
            self.stop = True
            self.thread.join()
            sys.setswitchinterval(self.switch)
            self.edges.append(self.nvml.sample())
            self.nvml.close()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def _smi_rows(self):
        rows = []
        if self.tmp is None:
            return rows
        self.tmp.flush()
        with open(self.tmp.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                             "sw_power_cap"]
                    rows.append((float(parts[1]),
                                 float(parts[2]) if parts[2].replace(".", "").isdigit() else 0.0,
                                 [names[i] for i in range(4) if parts[5 + i] == "Active"]))
        os.unlink(self.tmp.name)
        return rows

    def summary(self) -> dict:
        rows = (self.rows or self.edges) if self.nvml is not None else self._smi_rows()
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0,
                    "source": self.source}
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted({n for r in rows for n in r[2]}),
                "samples": len(rows), "source": self.source}


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


def workload_config(work: str, params: list[dict], precision: str) -> dict:
    """The workload as both arms name it (the GPU arm adds how it ran under
    "run")."""
    return {"workload": work, "lattices": [f"{p['nx']}x{p['ny']}" for p in params],
            "sims_per_gpu": len(params),
            "fluid_nodes_per_step": sum(fluid_nodes(p) for p in params),
            "physics": "density ratio 10, SRF quadratic law, Gibbs term (seeded synthetic)",
            "l2": l2_note(params, precision)}


def l2_note(params: list[dict], precision: str) -> str:
    """Working set (both population buffers of every simulation) against the
    129 MB L2: above it, every step streams its inputs from HBM."""
    mb = sum(2 * BYTES_PER_NODE_BUFFER[precision] * p["nx"] * p["ny"] for p in params) / 1e6
    if mb > 129.0:
        return "working set %.0f MB > 129 MB L2; simulations interleaved per step" % mb
    return "working set %.0f MB fits the 129 MB L2 (a profiling case, not a bench line)" % mb


def run_reference(args, budget_s: float = 150.0) -> None:
    """The oracle as the reference arm: each benchmark step advances lattices
    of the workload by one FP64 time step on the host cores -- all of them
    while the whole run fits about budget_s seconds, else a round-robin
    sample of them per step (every lattice is visited in turn)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    work = workload(args.workload)
    from oracle import oracle as orc
    threads = os.cpu_count() or 1
    used = orc.set_threads(threads)
    sims = []
    for p in work:
        o = orc.Oracle(p)
        o.init_fields(si.bubble_fields(p))
        sims.append(o)
    # calibration (untimed): one step of the first lattice
    t0 = time.perf_counter()
    sims[0].step(1)
    per_lattice = time.perf_counter() - t0
    per_step = max(1, min(len(sims), int(budget_s / max((args.steps + args.warmup) * per_lattice,
                                                         1e-9))))
    order = [i % len(sims) for i in range((args.steps + args.warmup) * per_step)]
    nodes = 0
    k = 0
    for _ in range(args.warmup):
        for _ in range(per_step):
            sims[order[k]].step(1)
            k += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(per_step):
            i = order[k]
            sims[i].step(1)
            nodes += fluid_nodes(work[i])
            k += 1
    dt = time.perf_counter() - t0
    for o in sims:
        o.close()
    v = nodes / dt / 1e6
    sample = (f"{args.steps} benchmark steps of {per_step} FP64 lattice step(s) each "
              f"(round robin over the {len(sims)} lattices of the workload) after "
              f"{args.warmup} warm-up steps, {dt:.1f} s")
    print(json.dumps({
        "impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / max(args.steps, 1) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.workload, work, args.precision),
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": used, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------- GPU arm
class Batch:
    """Simulations of one workload on one stream, stepped batched or plain."""

    def __init__(self, lbm, torch, params, precision, stream):
        self.lbm, self.torch, self.stream = lbm, torch, stream
        self.params = [dict(p, precision=PRECISION_CODE[precision]) for p in params]
        self.sims = [lbm.Sim(p, stream=stream, workspace="torch") for p in self.params]
        for s in self.sims:
            s.init()                      # analytic initial state, built on the device
        self.nodes = sum(fluid_nodes(p) for p in self.params)
        self.tuned_steps = 0

    def tune(self, steps):
        if steps > 0:
            self.tuned_steps += self.lbm.lbm_tune_batch(self.sims, steps)

    def launches(self):
        return sum(s.launches() for s in self.sims)

    def run(self, mode, nsteps, per_step=False, graph=False):
        if mode == "batched" and not per_step:
            self.lbm.lbm_step_batch(self.sims, nsteps)  # one call; runs of 64 replay graphs
        elif mode == "plain" and graph:
            for s in self.sims:                        # all steps of a sim in one call
                s.step(nsteps)
        else:
            for _ in range(nsteps):
                if mode == "batched":
                    self.lbm.lbm_step_batch(self.sims, 1)
                else:
                    for s in self.sims:
                        s.step(1)

    def timed(self, mode, nsteps, barrier, per_step=False, graph=False):
        """Device time (CUDA events on the sims' stream) of nsteps steps and
        the kernel launches they issued."""
        torch = self.torch
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        l0 = self.launches()
        ev0.record(self.stream)
        self.run(mode, nsteps, per_step, graph)
        ev1.record(self.stream)
        barrier()
        return ev0.elapsed_time(ev1), self.launches() - l0

    def close(self):
        for s in self.sims:
            s.close()


def tile_shapes(lbm, sims) -> list[str]:
    """The streaming tile shapes (columns x chunk rows) of a batch's plan."""
    return sorted({f"{w}x{h}" for w, h in lbm.lbm_batch_tiles(sims) if w})


# lbm_step_batch replays a graph for every 64 steps of a call and for a
# remainder of at least this many steps; lbm_step only for the 64-step runs
GRAPH_MIN_STEPS = 8


def launch_mode(mode, steps, per_step, graph):
    """How the timed steps were issued: "graph" when captured graphs
    replayed them (all of them, or all but a remainder of fewer than
    GRAPH_MIN_STEPS single launches)."""
    if mode == "batched":
        return "batched" + (" graph" if not per_step and steps >= GRAPH_MIN_STEPS else "")
    return "plain" + (" graph" if graph and steps >= 64 else "")


def warm_remainder(batch, steps: int) -> int:
    """A batched call of `steps` steps replays its own graph for the
    remainder of steps mod 64 (when at least GRAPH_MIN_STEPS): capture it
    before the timed region, from the buffers the timed call starts from
    (twice for an odd remainder, so that they return).  Returns the steps
    run."""
    rem = steps % 64
    if rem < GRAPH_MIN_STEPS:
        return 0
    n = 2 if rem % 2 else 1
    for _ in range(n):
        batch.run("batched", rem)
    return n * rem


def sub_measure(lbm, torch, dev_index, params, precision, mode, steps, tune_steps, stream,
                barrier, graph=True) -> dict:
    """A device-timed measurement of another workload or storage format, with
    its clocks: MLUPS and the fraction of the HBM roofline."""
    b = Batch(lbm, torch, params, precision, stream)
    if mode == "batched":
        b.tune(tune_steps)
        b.run(mode, 64)                   # warm-up that captures the batch graph
        warm_remainder(b, steps)
    else:
        b.run(mode, 64, graph=graph)
    with ClockSampler(dev_index) as clk:
        ms, launches = b.timed(mode, steps, barrier, graph=graph)
    c = clk.summary()
    value = b.nodes * steps / (ms * 1e-3) / 1e6
    gbs = value * 1e6 * BYTES_PER_NODE_STEP[precision] / 1e9
    peak = measured_peaks()["hbm_gbs"]
    out = {"value": value, "unit": "MLUPS", "storage": precision, "mode": mode,
           "launch_mode": launch_mode(mode, steps, False, graph),
           "lattices": sorted({f"{p['nx']}x{p['ny']}" for p in params}),
           "sims": len(params), "steps": steps, "gpu_launches": launches,
           "achieved_gbs": gbs, "hbm_frac": gbs / peak,
           "bytes_per_node_step": BYTES_PER_NODE_STEP[precision],
           "strip_chunks": sorted(set(lbm.lbm_batch_plan(b.sims)) - {0}),
           "tile_shapes": tile_shapes(lbm, b.sims),
           "clocks": {"sm_mhz": c["sm_mhz"], "reasons": c["reasons"], "samples": c["samples"]}}
    b.close()
    return out


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
    params = [dict(p, precision=PRECISION_CODE[args.precision]) for p in workload(args.workload)]
    batch = Batch(lbm, torch, params, args.precision, stream)
    nodes_per_step = batch.nodes
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # measured strip plan of the batched launch (steps outside the timed region)
    if args.mode == "batched":
        batch.tune(args.tune_steps)
    plan = lbm.lbm_batch_plan(batch.sims)
    tiles = tile_shapes(lbm, batch.sims)
    warmup_run = args.warmup
    batched_call = args.mode == "batched" and not args.per_step_calls
    if batched_call and args.steps >= 64:
        # at least one 64-step run, so that the batch's graph is captured
        # before the timed region
        warmup_run = max(args.warmup, 64)
    batch.run(args.mode, warmup_run, args.per_step_calls, args.graph)
    if batched_call:
        warmup_run += warm_remainder(batch, args.steps)
    with ClockSampler(dev_index) as clk:
        ms, launches = batch.timed(args.mode, args.steps, barrier, args.per_step_calls, args.graph)
    clocks = clk.summary()

    ms_max = max_over_ranks(ms, "cuda")
    value = weak_scaling_value(ms_max, nodes_per_step, args.steps, ws)

    # roofline of the dominant kernel: every launch in the timed region is a
    # fused step kernel (one simulation, or as many simulations of the batch
    # as one launch of the kernel family takes), so the algorithmic bytes of
    # one launch are those of all timed steps over the launch count
    per_launch_ms = ms / launches
    bpn = BYTES_PER_NODE_STEP[args.precision]
    per_launch_bytes = bpn * nodes_per_step * args.steps / launches
    peaks = measured_peaks()
    achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
    kernel = step_kernel_name(args.mode, args.precision, params)
    traffic = profiled_traffic(args.workload, args.mode, args.precision, params)

    # the other launch mode on the same simulations, for comparison
    other = None
    if args.compare_modes and len(params) > 1:
        mode = "plain" if args.mode == "batched" else "batched"
        n_o = max(args.steps // 4, 1)
        ms_o, _ = batch.timed(mode, n_o, barrier)
        other = {"mode": mode, "launch_mode": launch_mode(mode, n_o, False, False),
                 "value": nodes_per_step * n_o / (ms_o * 1e-3) / 1e6}
    batch.close()

    # sub-results on one GPU: the mixed-precision batched ensemble against the
    # plain single-simulation path, and the large-lattice precision study
    extra = {}
    if ws == 1 and not args.no_extra:
        plain = sub_measure(lbm, torch, dev_index, [si.channel_256x1024()], "fp32", "plain",
                            args.extra_steps, 0, stream, barrier)
        ens = sub_measure(lbm, torch, dev_index, si.ensemble_channels(64, seed=0), "fp16",
                          "batched", args.extra_steps, args.tune_steps, stream, barrier)
        extra["mixed_precision"] = {
            "batched_fp16_ensemble": ens, "plain_fp32_single": plain,
            "ratio": ens["value"] / plain["value"],
            "target_ratio": 2.0,
            "note": "64 channels of uneven size (nx 128..512, multiples of 16; ny = 4 nx) at "
                    "binary16 storage in one lbm_step_batch call, against lbm_step on one "
                    "256x1024 FP32 channel"}
        extra["config3"] = {
            prec: sub_measure(lbm, torch, dev_index, [si.channel_1024x4096()], prec, "batched",
                              args.extra_steps, args.tune_steps, stream, barrier)
            for prec in ("fp32", "fp16", "bf16")}
        # the small 64x128 channel is launch-bound: its 2000 steps as lbm_step
        # issues them (64-step CUDA graphs)
        extra["config1"] = sub_measure(lbm, torch, dev_index, [si.channel_64x128()], "fp32",
                                       "plain", 2000, 0, stream, barrier)

    e2e = run_e2e(args, lbm, torch, stream, params) if not args.no_e2e else None
    plain_value = extra.get("mixed_precision", {}).get("plain_fp32_single", {}).get("value")
    served = None
    if args.serve_requests > 0 and ws == 1:
        # requests that reach their terminal state, then the config's own
        # lattice range and start at a step cap (throughput of the mix)
        served = run_served(args, torch, "reference_plane", args.serve_nx_max,
                            args.serve_max_steps, plain_value)
        if args.serve_throughput_steps > 0:
            extra["served_throughput"] = run_served(args, torch, "quarter", 512,
                                                    args.serve_throughput_steps, plain_value)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload)
    if rank == 0:
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args.workload, params, args.precision),
            "run": {"storage": args.precision,
                    "launch_mode": launch_mode(args.mode, args.steps, args.per_step_calls,
                                               args.graph),
                    "warmup_steps_run": warmup_run,
                    "other_mode": other,
                    "strip_plan": {"tuned": batch.tuned_steps > 0,
                                   "tuning_steps": batch.tuned_steps,
                                   "strip_chunks": sorted(set(plan) - {0}),
                                   "tile_shapes": tiles},
                    "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                         "frac_of_nominal_8tbs": achieved / 8000.0,
                         "traffic": traffic, "peak_source": peaks["source"],
                         "kernel": kernel, "bytes_per_node_step": bpn},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "served": served,
            "gpu_launches": launches,
            "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                       "reasons": clocks["reasons"], "samples": clocks["samples"],
                       "source": clocks["source"]},
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def run_served(args, torch, start: str, nx_max: int, max_steps: int,
               plain_value=None) -> dict:
    """The served workload: a Poisson stream of requests (uneven lattices,
    physics and storage precisions) through the serving loop, arrivals in
    wall time.  A request ends at its terminal state (|U| < 1e-6 at every
    observation over a window of t* = R/U_o) or at the step cap.  Reports the
    converged and capped counts, p50/p99 of arrival-to-finish latency over all
    requests and over each class (also per storage format), and aggregate
    MLUPS (also against the plain single-simulation rate when given)."""
    from paper_2408_00146_gb300.serve import LbmEngine, Server, requests_from_stream, summary

    stream = si.request_stream(n=args.serve_requests, rate=args.serve_rate, seed=0,
                               start=start, nx_range=(64, nx_max))
    reqs = requests_from_stream(stream, max_steps=max_steps, tol=1e-6)
    free, _total = torch.cuda.mem_get_info()
    budget = int(min(150e9, 0.8 * free))
    engine = LbmEngine()
    srv = Server(engine, budget_bytes=budget, round_steps=args.serve_round_steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = srv.run(reqs)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    out = summary(res, wall, srv.node_steps)
    out.update({"rate_per_s": args.serve_rate, "max_steps": max_steps,
                "tol": 1e-6, "terminal_window": "t* = R/U_o (at least two rounds)",
                "round_steps": args.serve_round_steps, "budget_gb": budget / 1e9,
                "peak_resident": srv.peak_resident, "peak_gb": srv.peak_bytes / 1e9,
                "fp16_requests": sum(p["precision"] == 1 for _, p in stream),
                "lattices": f"nx log-uniform 64..{nx_max} (x16), ny = 4 nx",
                "start": START_NOTE[start],
                "tile_shapes": sorted(f"{w}x{h}" for w, h in engine.tiles),
                "vs_plain": out["mlups"] / plain_value if plain_value else None})
    return out


START_NOTE = {
    "quarter": "bubble a quarter of the way along the channel (config physics; its "
               "equilibrium is 1e5-1e7 steps away, so every request ends at the cap)",
    "reference_plane": "clean bubble (beta = 0) on the reference-temperature plane, the SRF "
                       "equilibrium: requests end when the start-up flow has decayed below "
                       "tol for t* = R/U_o",
}


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
        lbm.lbm_observe_enqueue(sims)     # every sim's observables, one wait
        lbm.lbm_observe_collect(sims)
        d2h += 13 * 8 * len(sims)
        done += n
    for s, out in zip(sims, host_out):
        lbm.lbm_observe(s.handle, out)
        d2h += out.size * 4 + 13 * 8
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
    ap.add_argument("--extra-steps", type=int, default=200,
                    help="timed steps of each sub-result (mixed_precision, config3)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the mixed_precision and config3 sub-results")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=500,
                    help="requests of the served workload (0: skip it)")
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-max-steps", type=int, default=300000,
                    help="step cap of the served run to terminal state")
    ap.add_argument("--serve-throughput-steps", type=int, default=4000,
                    help="step cap of the served run over the full lattice range (0: skip)")
    ap.add_argument("--serve-round-steps", type=int, default=128)
    ap.add_argument("--serve-nx-max", type=int, default=128,
                    help="largest nx of the served run to terminal state")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
