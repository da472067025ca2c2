"""GPU test of lbm_reduce_observables_noalloc, the observables reduction for
callers that cannot allocate device memory where they call it (stream
capture, latency-critical loops that must not take cudaMalloc's device-wide
synchronisation, fully pre-budgeted device memory).  It keeps its block
partial sums in a fixed array inside the library instead of a workspace.

Checked through the C ABI against lbm_observe, the existing entry point that
reduces the same fields with workspace scratch: two calls in a row, so the
second call also shows that whatever the first left in the shared array does
not leak into the result.  Collected last on purpose (file name) so that a
run stopping at the first failure has run every other test first."""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu


def _noalloc_sums(lbm, torch, d_fields, p, stream):
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    lbm.lbm_reduce_observables_noalloc(d_fields.data_ptr(), p["nx"], p["ny"], p["walls"],
                                       out.data_ptr(), stream)
    stream.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("shape", [(64, 128, 1), (256, 1024, 1), (37, 29, 0)])
def test_noalloc_reduction_matches_observe(shape):
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2408_00146_gb300 import lbm

    nx, ny, walls = shape
    p = si.scaled_channel(nx, ny)
    p.update(walls=walls, R=max(min(nx, ny) / 5.0, 4.0), xb=nx / 2, yb=ny / 2)
    stream = torch.cuda.Stream()
    sim = lbm.Sim(p, stream=stream)
    sim.init(si.parity_fields(p, seed=5))
    sim.step(25)
    host = np.zeros((6, ny, nx))
    ref = lbm.lbm_observe(sim.handle, host)
    # the same FP32 field values, now in caller-owned device memory
    d_fields = torch.tensor(host, dtype=torch.float32, device="cuda")
    nodes = nx * (ny - 2 if walls else ny)
    for _ in range(2):
        s = _noalloc_sums(lbm, torch, d_fields, p, stream)
        assert s[7] == nodes and s[6] == 0
        assert s[0] == pytest.approx(ref["mass_phi"], rel=1e-12)
        assert s[1] == pytest.approx(ref["mass_psi"], rel=1e-12)
        assert s[2] / s[0] == pytest.approx(ref["xc"], rel=1e-12)
        assert s[3] / s[0] == pytest.approx(ref["yc"], rel=1e-12)
        assert s[4] / s[0] == pytest.approx(ref["ux_bub"], rel=1e-9, abs=1e-15)
        assert s[5] / s[0] == pytest.approx(ref["uy_bub"], rel=1e-9, abs=1e-15)
    sim.close()


def test_noalloc_rejects_lattices_beyond_its_scratch():
    import torch
    from paper_2408_00146_gb300 import lbm

    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        # 4097 x 4098 with walls: 4097 x 4096 = 16,781,312 fluid nodes > 16,777,216
        lbm.lbm_reduce_observables_noalloc(d.data_ptr(), 4097, 4098, 1, d.data_ptr(), None)
    assert e.value.status == lbm.LBM_EINVAL and "at most" in str(e.value)
