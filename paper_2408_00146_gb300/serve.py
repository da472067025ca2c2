"""Serving of many independent bubble-migration simulations on one GPU.

Requests (one parameter set each, arriving over time) are admitted while
their device workspaces fit a memory budget, kept resident, and advanced
together: every round steps all resident simulations by ``round_steps``
time steps with ``lbm_step_batch`` (one launch per step and kernel family for
up to 64 simulations).  Rounds are pipelined: the observables of every
resident simulation after a round are enqueued on the device
(``lbm_observe_enqueue``) and read (``lbm_observe_collect``) while the next
round runs, so the host's bookkeeping never leaves the GPU idle.

A simulation reaches its terminal state when its bubble velocity |U| (the
phi-weighted mean velocity of Sec. 6) has stayed below ``tol`` at every
observation over a window of at least one characteristic time t* = R/U_o
(Eq. (21)) and two rounds; a bubble that sloshes through U = 0 exceeds tol
within such a window and does not stop.  A simulation also stops at its step
cap.  Its memory is then released and waiting requests are admitted before
the next round (continuous batching).  Each simulation's trajectory is
independent of what else is resident, because a batched step computes every
simulation exactly as a step of its own would, and the decisions depend only
on its own observations.

The scheduler only orders work on the host; every step of every simulation
runs in the CUDA kernels behind the C ABI.  ``Server`` takes an engine
object so that its policy can be exercised without a GPU.
"""
from __future__ import annotations

import dataclasses
import math
import time
from collections import deque

MAX_BATCH = 64   # simulations per lbm_step_batch call (the C ABI's limit)


@dataclasses.dataclass
class Request:
    rid: int
    params: dict
    arrival: float = 0.0           # seconds after the start of the run
    max_steps: int = 300_000
    tol: float = 1e-6
    window_steps: int | None = None    # terminal window; None: max(t*, 2 rounds)


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    converged: bool
    status: str                    # "converged", "step cap" or an error
    obs: dict
    nodes: int
    storage: int = 0               # population storage: 0 FP32, 1 binary16, 2 bfloat16

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class LbmEngine:
    """Engine over the C ABI: workspaces from PyTorch's caching allocator
    (no cudaMalloc per request), all simulations on one stream."""

    def __init__(self, stream=None):
        import torch

        from . import lbm
        self.lbm = lbm
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.tiles: set[tuple[int, int]] = set()   # streaming tile shapes used

    def workspace_bytes(self, params: dict) -> int:
        return self.lbm.lbm_workspace_bytes(params)

    def open(self, params: dict):
        sim = self.lbm.Sim(params, stream=self.stream, workspace="torch")
        sim.init()                  # analytic initial state, built on the device
        return sim

    def step(self, sims: list, n: int) -> None:
        for i in range(0, len(sims), MAX_BATCH):
            batch = sims[i:i + MAX_BATCH]
            self.lbm.lbm_step_batch(batch, n)
            self.tiles.update(t for t in self.lbm.lbm_batch_tiles(batch) if t[0])

    def observe_enqueue(self, sims: list) -> None:
        for i in range(0, len(sims), MAX_BATCH):
            self.lbm.lbm_observe_enqueue(sims[i:i + MAX_BATCH])

    def observe_collect(self, sims: list) -> list[dict]:
        out = []
        for i in range(0, len(sims), MAX_BATCH):
            out += self.lbm.lbm_observe_collect(sims[i:i + MAX_BATCH])
        return out

    def close(self, sim) -> None:
        sim.close()


def fluid_nodes(p: dict) -> int:
    return int(p["nx"]) * (int(p["ny"]) - 2 if p.get("walls", 1) else int(p["ny"]))


class Server:
    """Admission by memory budget, resident state, continuous batching.

    clock: returns seconds; wait(dt): lets dt seconds pass when nothing is
    resident and the next request has not arrived yet.  Defaults are wall
    time; tests pass a virtual clock."""

    def __init__(self, engine, budget_bytes: int, round_steps: int = 100,
                 clock=time.perf_counter, wait=time.sleep):
        if round_steps < 1:
            raise ValueError("round_steps must be >= 1")
        self.engine = engine
        self.budget = int(budget_bytes)
        self.round_steps = int(round_steps)
        self.clock = clock
        self.wait = wait
        self.node_steps = 0
        self.rounds = 0
        self.peak_bytes = 0
        self.peak_resident = 0

    def window(self, req: Request, ob: dict) -> int:
        """Steps over which |U| must stay below tol: the request's own, else
        t* = R/U_o (from the observation) and at least two rounds."""
        if req.window_steps is not None:
            return int(req.window_steps)
        w = 2 * self.round_steps
        uo, R = ob.get("U_o", 0.0), float(req.params.get("R", 0.0))
        if uo > 0 and R > 0:
            w = max(w, int(math.ceil(R / uo)))
        return w

    def run(self, requests: list[Request]) -> list[Result]:
        for r in requests:
            if self.engine.workspace_bytes(r.params) > self.budget:
                raise ValueError(f"request {r.rid} needs more memory than the whole budget")
        pending = deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        waiting: list[Request] = []
        resident: dict[int, dict] = {}        # rid -> {req, sim, bytes, steps, admitted, ...}
        used = 0
        results: list[Result] = []
        inflight: list[tuple[int, int]] = []  # (rid, steps) of the enqueued observation
        t0 = self.clock()

        def now() -> float:
            return self.clock() - t0

        while pending or waiting or resident:
            t = now()
            while pending and pending[0].arrival <= t:
                waiting.append(pending.popleft())
            # admission: first fit in arrival order
            still = []
            for r in waiting:
                nbytes = self.engine.workspace_bytes(r.params)
                if used + nbytes <= self.budget:
                    used += nbytes
                    resident[r.rid] = dict(req=r, sim=self.engine.open(r.params), bytes=nbytes,
                                           steps=0, admitted=now(), last_fast=0)
                else:
                    still.append(r)
            waiting = still
            self.peak_bytes = max(self.peak_bytes, used)
            self.peak_resident = max(self.peak_resident, len(resident))
            if not resident:
                if pending:
                    self.wait(max(pending[0].arrival - now(), 0.0))
                continue
            # one round: every resident simulation advances round_steps steps
            order = sorted(resident)
            self.engine.step([resident[k]["sim"] for k in order], self.round_steps)
            self.rounds += 1
            for k in order:
                resident[k]["steps"] += self.round_steps
                self.node_steps += fluid_nodes(resident[k]["req"].params) * self.round_steps
            # the previous round's observables, read while this round runs
            live = [(k, st) for k, st in inflight if k in resident]
            obs = self.engine.observe_collect([resident[k]["sim"] for k, _ in live]) if live else []
            for (k, st), ob in zip(live, obs):
                ent = resident[k]
                req = ent["req"]
                u = math.hypot(ob["ux_bub"], ob["uy_bub"])
                status = None
                if ob.get("status", 0) != 0 or not math.isfinite(u):
                    status = f"error {ob.get('status', 0)}"
                else:
                    if u >= req.tol:
                        ent["last_fast"] = st
                    if st - ent["last_fast"] >= self.window(req, ob):
                        status = "converged"
                    elif st >= req.max_steps:
                        status = "step cap"
                if status is None:
                    continue
                self.engine.close(ent["sim"])
                used -= ent["bytes"]
                results.append(Result(rid=req.rid, arrival=req.arrival, admitted=ent["admitted"],
                                      finished=now(), steps=st, converged=status == "converged",
                                      status=status, obs=dict(ob),
                                      nodes=fluid_nodes(req.params),
                                      storage=int(req.params.get("precision", 0))))
                del resident[k]
            # observables after this round, collected during the next one
            order = sorted(resident)
            if order:
                self.engine.observe_enqueue([resident[k]["sim"] for k in order])
            inflight = [(k, resident[k]["steps"]) for k in order]
        return sorted(results, key=lambda r: r.rid)


def percentile(values: list[float], q: float) -> float:
    """q-th percentile (0..100) by linear interpolation between order
    statistics."""
    if not values:
        return float("nan")
    v = sorted(values)
    pos = (len(v) - 1) * q / 100.0
    lo = int(math.floor(pos))
    hi = min(lo + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (pos - lo)


STORAGE_NAMES = {0: "fp32", 1: "fp16", 2: "bf16"}


def _classes(results: list[Result]) -> dict:
    conv = [r.latency for r in results if r.converged]
    cap = [r.latency for r in results if r.status == "step cap"]
    steps = [r.steps for r in results if r.converged]
    return {"requests": len(results), "converged": len(conv), "capped": len(cap),
            "errors": len(results) - len(conv) - len(cap),
            "p50_converged_s": percentile(conv, 50.0), "p99_converged_s": percentile(conv, 99.0),
            "p50_capped_s": percentile(cap, 50.0), "p99_capped_s": percentile(cap, 99.0),
            "p50_steps_to_terminal": percentile(steps, 50.0)}


def summary(results: list[Result], wall_s: float, node_steps: int) -> dict:
    """Latency percentiles over all requests, and separately over those that
    reached their terminal state and those stopped by the step cap; the same
    split per population storage format."""
    lat = [r.latency for r in results]
    out = _classes(results)
    out.pop("requests")
    by = {}
    for code, name in STORAGE_NAMES.items():
        sub = [r for r in results if r.storage == code]
        if sub:
            by[name] = _classes(sub)
    return {"requests": len(results), **{k: out[k] for k in ("converged", "capped", "errors")},
            "p50_latency_s": percentile(lat, 50.0), "p99_latency_s": percentile(lat, 99.0),
            **{k: v for k, v in out.items() if k not in ("converged", "capped", "errors")},
            "by_storage": by,
            "mlups": node_steps / wall_s / 1e6 if wall_s > 0 else float("nan"),
            "wall_s": wall_s}


def requests_from_stream(stream: list[tuple[float, dict]], max_steps: int,
                         tol: float = 1e-6) -> list[Request]:
    return [Request(rid=i, params=p, arrival=t, max_steps=max_steps, tol=tol)
            for i, (t, p) in enumerate(stream)]
