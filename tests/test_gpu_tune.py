"""Strip plans of the batched streaming launch: the plan lbm_step_batch uses
(lbm_batch_plan) and its measured choice (lbm_tune_batch).  A step's result
does not depend on the plan, so a tuned batch must hold exactly the
populations of a batch stepped the same number of times without tuning."""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2408_00146_gb300 import lbm as L
    L.load()
    return L


def _mix():
    """Three FP32 streaming lattices of different heights (80 x 66 with a
    partial last column of 16 nodes; 32 x 290), one FP32 tile-kernel lattice
    (nx = 45: no 16-byte TMA rows), one binary16 tile-kernel lattice (nx = 60)
    and binary16 and bfloat16 streaming lattices (launches of their own)."""
    ps = [si.scaled_channel(64, 160), si.scaled_channel(80, 66), si.scaled_channel(32, 290),
          si.scaled_channel(45, 64), si.scaled_channel(60, 96), si.scaled_channel(48, 80),
          si.scaled_channel(40, 72)]
    ps[4]["precision"] = 1
    ps[5]["precision"] = 1
    ps[6]["precision"] = 2
    for p in ps:
        p["R"] = min(p["R"], 8.0)
    return ps


def _sims(lbm, ps, stream):
    sims = [lbm.Sim(p, stream=stream) for p in ps]
    for i, (s, p) in enumerate(zip(sims, ps)):
        s.init(si.parity_fields(p, seed=40 + i))
    return sims


def test_plan_reports_streaming_and_tile_sims(lbm):
    import torch
    ps = _mix()
    sims = _sims(lbm, ps, torch.cuda.Stream())
    plan = lbm.lbm_batch_plan(sims)
    assert len(plan) == len(ps)
    assert all(c >= 4 for c in plan[:3]) and plan[3] == 0 and plan[4] == 0
    assert plan[5] >= 4 and plan[6] >= 4
    assert lbm.lbm_batch_plan(sims) == plan          # cached: the same answer again


def test_tuned_batch_equals_untuned_batch(lbm):
    import torch
    ps = _mix()
    st = torch.cuda.Stream()
    tuned, plain = _sims(lbm, ps, st), _sims(lbm, ps, st)
    taken = lbm.lbm_tune_batch(tuned, 2)
    # one warm-up step and two per distinct candidate plan
    assert taken >= 3 and (taken - 1) % 2 == 0
    lbm.lbm_step_batch(plain, taken)
    for a, b in zip(tuned, plain):
        assert a.observe()["t"] == b.observe()["t"] == taken
        assert np.array_equal(a.populations(), b.populations())
    # the tuned plan is what later batch steps use, and it keeps the result
    plan = lbm.lbm_batch_plan(tuned)
    assert all(c >= 4 for c in plan[:3]) and plan[3:5] == [0, 0]
    assert plan[5] >= 4 and plan[6] >= 4
    lbm.lbm_step_batch(tuned, 5)
    lbm.lbm_step_batch(plain, 5)
    for a, b in zip(tuned, plain):
        assert np.array_equal(a.populations(), b.populations())


def test_tune_without_streaming_sims_and_bad_arguments(lbm):
    import torch
    st = torch.cuda.Stream()
    tile_only = _sims(lbm, [si.scaled_channel(45, 64)], st)
    assert lbm.lbm_tune_batch(tile_only, 3) == 0
    assert tile_only[0].observe()["t"] == 0
    sims = _sims(lbm, _mix()[:2], st)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_tune_batch(sims, 0)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_tune_batch([sims[0], sims[0]], 1)
    assert sims[0].observe()["t"] == 0


def test_graph_replayed_batch_equals_single_steps(lbm):
    """lbm_step_batch replays a captured graph for runs of 64 steps; its
    result and launch count equal those of the same steps issued one call
    at a time, with the sims starting from different buffers and a graph
    taken again from the cache."""
    import torch
    ps = _mix()
    st = torch.cuda.Stream()
    a, b = _sims(lbm, ps, st), _sims(lbm, ps, st)
    a[1].step(1)
    b[1].step(1)
    l0a, l0b = a[0].launches(), b[0].launches()
    lbm.lbm_step_batch(a, 130)
    for _ in range(130):
        lbm.lbm_step_batch(b, 1)
    assert a[0].launches() - l0a == b[0].launches() - l0b
    for x, y in zip(a, b):
        assert np.array_equal(x.populations(), y.populations())
    lbm.lbm_step_batch(a, 64)
    lbm.lbm_step_batch(b[:2], 64)       # another batch in between
    lbm.lbm_step_batch(b[2:], 64)
    for x, y in zip(a, b):
        assert np.array_equal(x.populations(), y.populations())
        assert x.observe()["t"] == y.observe()["t"]
