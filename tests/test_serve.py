"""Serving loop: admission by memory budget, continuous batching, latency
statistics (host policy with a fake engine, no GPU), and on the GPU that a
request's result alone equals its result in a mix."""
import math

import numpy as np
import pytest

import seeded_inputs as si
from paper_2408_00146_gb300.serve import Request, Server, percentile, summary


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def wait(self, dt):
        self.t += dt


class FakeEngine:
    """Simulations whose bubble velocity halves every step from U0 = 1e-3;
    each round costs one unit of virtual time.  Observations are enqueued
    (the state is recorded) and collected later, as on the device."""

    def __init__(self, clock):
        self.clock = clock
        self.open_now = 0
        self.max_open = 0
        self.log = []

    def workspace_bytes(self, p):
        return p["nx"] * p["ny"]

    def open(self, p):
        self.open_now += 1
        self.max_open = max(self.max_open, self.open_now)
        return {"p": p, "t": 0, "seen": None}

    def step(self, sims, n):
        self.log.append(len(sims))
        self.clock.t += 1.0
        for s in sims:
            s["t"] += n

    def velocity(self, t):
        return 1e-3 * 0.5 ** t

    def observe_enqueue(self, sims):
        for s in sims:
            s["seen"] = s["t"]

    def observe_collect(self, sims):
        return [{"ux_bub": 0.0, "uy_bub": self.velocity(s["seen"]), "status": 0,
                 "yc": float(s["seen"])} for s in sims]

    def close(self, s):
        self.open_now -= 1


class StartupEngine(FakeEngine):
    """The bubble starts at rest: |U| = 0 until step 10, then 1e-3 halving
    every step."""

    def velocity(self, t):
        return 0.0 if t < 10 else 1e-3 * 0.5 ** (t - 10)


class SloshEngine(FakeEngine):
    """A bubble oscillating about its equilibrium: U = 1e-3 cos(2 pi t / 40),
    which is sampled exactly at a zero crossing every 20 steps."""

    def velocity(self, t):
        return abs(1e-3 * math.cos(2.0 * math.pi * t / 40.0))


def _req(rid, nx, arrival=0.0, tol=1e-9, max_steps=1000):
    p = si.scaled_channel(nx, 4 * nx)
    return Request(rid=rid, params=p, arrival=arrival, tol=tol, max_steps=max_steps)


def test_budget_and_continuous_batching():
    clk = FakeClock()
    eng = FakeEngine(clk)
    # budget for two 64x256 requests at a time
    budget = 2 * 64 * 256
    reqs = [_req(i, 64) for i in range(5)]
    srv = Server(eng, budget, round_steps=5, clock=clk, wait=clk.wait)
    res = srv.run(reqs)
    assert [r.rid for r in res] == list(range(5))
    assert eng.max_open == 2 and srv.peak_bytes <= budget
    # 1e-3 * 2^-t < 1e-9 first at t = 20; |U| < tol over a window of two
    # rounds (10 steps) after the last fast observation (t = 15) holds at
    # t = 25, which is read one round later (pipelined rounds)
    assert all(r.steps == 25 and r.converged for r in res)
    # admitted in arrival order as slots free: 0,1 at t=0; 2,3 after 6
    # rounds; 4 after 12 rounds
    adm = [r.admitted for r in res]
    assert adm == [0.0, 0.0, 6.0, 6.0, 12.0]
    assert eng.log == [2] * 12 + [1] * 6
    assert srv.node_steps == 5 * 30 * 64 * 254


def test_first_fit_admission_and_arrivals():
    clk = FakeClock()
    eng = FakeEngine(clk)
    big, small = _req(0, 128), _req(1, 64, arrival=0.5)
    late = _req(2, 64, arrival=10.0)
    budget = 128 * 512 + 64 * 256      # the big one and one small one fit together
    srv = Server(eng, budget, round_steps=10, clock=clk, wait=clk.wait)
    res = srv.run([late, small, big])
    by = {r.rid: r for r in res}
    assert by[0].admitted == 0.0
    assert by[1].admitted == 1.0          # arrives during round 1, admitted after it
    assert by[2].admitted >= 10.0         # the server waits for the late arrival
    assert by[2].latency == pytest.approx(by[2].finished - 10.0)
    assert all(r.status == "converged" for r in res)


def test_step_cap_and_oversized_request():
    clk = FakeClock()
    eng = FakeEngine(clk)
    srv = Server(eng, 10 ** 9, round_steps=7, clock=clk, wait=clk.wait)
    (r,) = srv.run([_req(0, 64, tol=0.0, max_steps=20)])
    assert r.status == "step cap" and not r.converged and r.steps == 21
    with pytest.raises(ValueError):
        Server(eng, 100, clock=clk, wait=clk.wait).run([_req(1, 64)])


def test_rest_shorter_than_the_window_is_not_terminal():
    clk = FakeClock()
    srv = Server(StartupEngine(clk), 10 ** 9, round_steps=5, clock=clk, wait=clk.wait)
    (r,) = srv.run([_req(0, 64, tol=1e-9)])
    # at rest for 5 steps (< the 10-step window); moving from t = 10, fast
    # until t = 25, below tol at t = 30 and 35
    assert r.converged and r.steps == 35


def test_sloshing_bubble_does_not_pass_the_terminal_test():
    """|U| sampled at a zero crossing (every 20 steps) is below tol, but the
    samples between are not: only the step cap stops it."""
    clk = FakeClock()
    srv = Server(SloshEngine(clk), 10 ** 9, round_steps=10, clock=clk, wait=clk.wait)
    (r,) = srv.run([_req(0, 64, tol=1e-6, max_steps=400)])
    assert r.status == "step cap" and r.steps == 400


def test_window_is_one_characteristic_time():
    """Without a request window the terminal window is t* = R/U_o from the
    observation (Eq. (21)), and at least two rounds."""
    srv = Server(FakeEngine(FakeClock()), 10 ** 9, round_steps=100)
    req = _req(0, 64)
    assert srv.window(req, {"U_o": req.params["R"] / 5000.0}) == 5000
    assert srv.window(req, {"U_o": 1.0}) == 200
    assert srv.window(req, {}) == 200
    req.window_steps = 30
    assert srv.window(req, {"U_o": 1e-3}) == 30


def test_error_status_finishes_request():
    clk = FakeClock()
    eng = FakeEngine(clk)
    eng.observe_collect = lambda sims: [{"ux_bub": math.nan, "uy_bub": 0.0, "status": -4}
                                        for _ in sims]
    srv = Server(eng, 10 ** 9, clock=clk, wait=clk.wait)
    (r,) = srv.run([_req(0, 64)])
    assert r.status.startswith("error") and not r.converged


def test_percentile_matches_linear_interpolation():
    rng = np.random.default_rng(0)
    v = list(rng.exponential(size=101))
    for q in (0, 1, 50, 99, 100):
        assert percentile(v, q) == pytest.approx(float(np.percentile(v, q)))
    s = summary([], 1.0, 0)
    assert s["requests"] == 0 and math.isnan(s["p50_latency_s"])
    assert s["converged"] == s["capped"] == s["errors"] == 0


def test_summary_splits_by_storage():
    from paper_2408_00146_gb300.serve import Result
    mk = lambda rid, lat, conv, st: Result(rid=rid, arrival=0.0, admitted=0.0, finished=lat,
                                           steps=100 * rid, converged=conv,
                                           status="converged" if conv else "step cap",
                                           obs={}, nodes=1, storage=st)
    res = [mk(1, 1.0, True, 0), mk(2, 3.0, True, 0), mk(3, 9.0, False, 1), mk(4, 2.0, True, 1)]
    s = summary(res, 1.0, 0)
    assert (s["converged"], s["capped"], s["errors"]) == (3, 1, 0)
    assert s["p50_converged_s"] == 2.0 and s["p50_capped_s"] == 9.0
    assert s["by_storage"]["fp32"]["converged"] == 2 and s["by_storage"]["fp32"]["capped"] == 0
    assert s["by_storage"]["fp16"]["capped"] == 1
    assert s["by_storage"]["fp16"]["p50_steps_to_terminal"] == 400
    assert "bf16" not in s["by_storage"]


def test_request_stream_shapes():
    st = si.request_stream(n=200, rate=20.0, seed=3)
    t = np.array([a for a, _ in st])
    assert np.all(np.diff(t) > 0)
    assert abs(t[-1] / 200 - 1 / 20.0) < 0.02          # mean gap 1/rate
    nx = np.array([p["nx"] for _, p in st])
    assert nx.min() >= 64 and nx.max() <= 512 and np.all(nx % 16 == 0)
    assert all(p["ny"] == 4 * p["nx"] for _, p in st)
    assert 0.3 < np.mean([p["precision"] for _, p in st]) < 0.7


@pytest.mark.gpu
def test_result_alone_equals_result_in_the_mix():
    """A request's final observables and step count are the same whether it
    runs alone or batched with others of other sizes and precisions, with
    admission delayed by the budget."""
    import torch
    assert torch.cuda.is_available()
    from paper_2408_00146_gb300 import lbm
    from paper_2408_00146_gb300.serve import LbmEngine

    stream = si.request_stream(n=6, rate=1e9, seed=5, nx_range=(64, 160))
    reqs = [Request(rid=i, params=p, arrival=0.0, max_steps=300, tol=1e-12)
            for i, (_, p) in enumerate(stream)]
    # the observation reaching the 300-step cap is read one round later
    eng = LbmEngine()
    ws = [lbm.lbm_workspace_bytes(r.params) for r in reqs]
    mix = Server(eng, budget_bytes=sum(sorted(ws)[-3:]), round_steps=100).run(reqs)
    assert len(mix) == len(reqs)
    for r in reqs:
        (alone,) = Server(LbmEngine(), budget_bytes=ws[r.rid], round_steps=100).run([r])
        m = mix[r.rid]
        assert m.steps == alone.steps == 300
        for k in ("xc", "yc", "ux_bub", "uy_bub", "mass_phi", "mass_psi"):
            assert m.obs[k] == alone.obs[k], (r.rid, k)
