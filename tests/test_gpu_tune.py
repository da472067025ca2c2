"""Strip plans of the batched streaming launch: the plan lbm_step_batch uses
(lbm_batch_plan, lbm_batch_tiles), its measured choice (lbm_tune_batch) and a
plan set by the caller (lbm_pin_batch_plan).  A step's result does not depend
on the plan -- tile shape and strip length -- so a tuned batch must hold
exactly the populations of a batch stepped the same number of times without
tuning, and the two compiled tile shapes must give identical steps."""
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


def test_tile_shapes_give_identical_steps(lbm):
    """The 32 x 8 and 64 x 4 tile shapes (the second for FP32 storage only),
    pinned on the same lattices (partial last columns of 16 and 32 nodes,
    beside 16-bit streaming and tile-kernel lattices), step bit for bit
    alike."""
    import torch
    ps = _mix()
    st = torch.cuda.Stream()
    a, b = _sims(lbm, ps, st), _sims(lbm, ps, st)
    streaming = [c > 0 for c in lbm.lbm_batch_plan(a)]
    fp32 = [p.get("precision", 0) == 0 for p in ps]
    wide = [64 if f else 32 for f in fp32]
    # plans are kept per list of lattice sizes: pin, step, then pin the other
    lbm.lbm_pin_batch_plan(a, [32] * len(ps), [6] * len(ps))
    assert lbm.lbm_batch_tiles(a) == [(32, 8) if s else (0, 0) for s in streaming]
    lbm.lbm_step_batch(a, 70)        # one captured 64-step graph and single steps
    lbm.lbm_pin_batch_plan(b, wide, [9] * len(ps))
    assert lbm.lbm_batch_tiles(b) == [((64, 4) if f else (32, 8)) if s else (0, 0)
                                      for s, f in zip(streaming, fp32)]
    assert [c for c, s in zip(lbm.lbm_batch_plan(b), streaming) if s] == [9] * sum(streaming)
    lbm.lbm_step_batch(b, 70)
    for x, y in zip(a, b):
        assert np.array_equal(x.populations(), y.populations())


def test_tuned_plan_names_its_tile_shape(lbm):
    import torch
    ps = _mix()
    sims = _sims(lbm, ps, torch.cuda.Stream())
    lbm.lbm_tune_batch(sims, 1)
    tiles = lbm.lbm_batch_tiles(sims)
    plan = lbm.lbm_batch_plan(sims)
    for (w, h), c in zip(tiles, plan):
        assert (w, h) in ((32, 8), (64, 4)) if c > 0 else (w, h) == (0, 0)
    # one shape per streaming launch; the 16-bit launches in 32 x 8
    assert len({tiles[i] for i in range(3)}) == 1
    assert tiles[5] == tiles[6] == (32, 8)


def test_pin_rejects_bad_plans(lbm):
    import torch
    sims = _sims(lbm, _mix()[:3], torch.cuda.Stream())
    for w, c in (([48] * 3, [8] * 3), ([32] * 3, [0] * 3), ([32, 64, 32], [8] * 3)):
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_pin_batch_plan(sims, w, c)
        assert ei.value.status == lbm.LBM_EINVAL
    # 64 x 4 has no 16-bit kernels
    s16 = _sims(lbm, _mix()[5:6], torch.cuda.Stream())
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_pin_batch_plan(s16, [64], [8])
    assert ei.value.status == lbm.LBM_EINVAL


def test_tile_shapes_identical_at_full_size(lbm):
    """The largest lattice of the benchmarks, 1024 x 4096 (FP32), steps bit for
    bit alike in the 32 x 8 and 64 x 4 tile shapes."""
    import torch
    p = si.channel_1024x4096()
    st = torch.cuda.Stream()
    a, b = lbm.Sim(p, stream=st), lbm.Sim(p, stream=st)
    f = si.parity_fields(p, seed=3)
    a.init(f)
    b.init(f)
    lbm.lbm_pin_batch_plan([a], [32], [57])
    lbm.lbm_step_batch([a], 3)
    lbm.lbm_pin_batch_plan([b], [64], [64])
    assert lbm.lbm_batch_tiles([b]) == [(64, 4)]
    lbm.lbm_step_batch([b], 3)
    assert np.array_equal(a.populations(), b.populations())
    a.close()
    b.close()


def test_short_graph_runs_equal_single_steps(lbm):
    """Batched calls of 8 to 63 steps replay a graph of their own once it is
    captured; odd and even lengths, replayed twice, equal single steps."""
    import torch
    ps = _mix()
    st = torch.cuda.Stream()
    a, b = _sims(lbm, ps, st), _sims(lbm, ps, st)
    l0a, l0b = a[0].launches(), b[0].launches()
    for n in (20, 20, 13, 13, 7):
        lbm.lbm_step_batch(a, n)
        for _ in range(n):
            lbm.lbm_step_batch(b, 1)
    assert a[0].launches() - l0a == b[0].launches() - l0b
    for x, y in zip(a, b):
        assert x.observe()["t"] == y.observe()["t"] == 73
        assert np.array_equal(x.populations(), y.populations())
