"""Host-side checks of the C-ABI library (no GPU needed): it builds for
sm_103a, loads, exports every entry point include/lbm.h declares, and its
host-only parameter handling agrees with the oracle's."""
import ctypes
import os
import re

import pytest

import seeded_inputs as si

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    with open(os.path.join(ROOT, "include", "lbm.h")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    for m in re.finditer(r"\b(lbm_[a-z_]+)\s*\(", src):
        names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2408_00146_gb300 import lbm
    L = lbm.load()
    declared = _declared()
    assert declared == set(lbm.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name


def test_library_is_built_for_sm103a():
    from paper_2408_00146_gb300 import build
    path = build.build()
    with open(path, "rb") as fh:
        blob = fh.read()
    assert b"sm_103a" in blob or b"compute_103a" in blob


@pytest.mark.parametrize("cfg", ["64x128", "256x1024", "1024x4096", "periodic"])
def test_derived_parameters_match_oracle(orc, cfg):
    from paper_2408_00146_gb300 import lbm
    p = {"64x128": si.channel_64x128(), "256x1024": si.channel_256x1024(0.2, 2e-3),
         "1024x4096": si.channel_1024x4096(), "periodic": si.channel_64x128()}[cfg]
    if cfg == "periodic":
        p.update(walls=0, sigma_TT=0.0, nu_A=0.2, alpha_A=0.05)
    a = lbm.lbm_derive(p)
    b = orc.derive(p)
    for k, v in b.items():
        assert a[k] == pytest.approx(v, rel=1e-14, abs=1e-300), k


@pytest.mark.parametrize("bad", [
    dict(nx=3), dict(ny=4), dict(M_phi=-0.1), dict(R=40.0), dict(W=0.0),
    dict(precision=7), dict(sigma_TT=0.0), dict(walls=2), dict(nx=100000, ny=100000),
    dict(psi_bc=3), dict(psi_bc=-1), dict(psi_bc=1, psi_L=1.0), dict(psi_bc=2, psi_R=-0.5),
])
def test_invalid_parameters_rejected(bad):
    from paper_2408_00146_gb300 import lbm
    p = si.channel_64x128()
    p.update(bad)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_derive(p)
    assert ei.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError):
        lbm.lbm_workspace_bytes(p)


def test_workspace_bytes_layout():
    from paper_2408_00146_gb300 import lbm
    p = si.channel_256x1024()
    n = p["nx"] * p["ny"]
    ws = lbm.lbm_workspace_bytes(p)
    # two population buffers (36 floats/node) + fields (6 floats/node) + scratch
    assert ws >= (2 * 36 + 6) * 4 * n
    assert ws < (2 * 36 + 6) * 4 * n + 64 * 1024
    # 16-bit storage: per buffer 36 two-byte deviations + a float4 of rest
    # moments per node
    for prec in (lbm.LBM_FP16, lbm.LBM_BF16):
        q = dict(p, precision=prec)
        ws16 = lbm.lbm_workspace_bytes(q)
        assert ws16 >= (2 * (36 * 2 + 16) + 6 * 4) * n
        assert ws16 < (2 * (36 * 2 + 16) + 6 * 4) * n + 64 * 1024
        assert lbm.lbm_derive(q)["U_o"] == lbm.lbm_derive(p)["U_o"]


def test_batch_calls_reject_empty_batches_on_the_host():
    """Argument checks of the batch entry points run before any CUDA call."""
    from paper_2408_00146_gb300 import lbm
    for call in (lambda: lbm.lbm_step_batch([], 1), lambda: lbm.lbm_tune_batch([], 1),
                 lambda: lbm.lbm_batch_plan([]), lambda: lbm.lbm_batch_tiles([]),
                 lambda: lbm.lbm_pin_batch_plan([], [], []),
                 lambda: lbm.lbm_observe_enqueue([]), lambda: lbm.lbm_observe_collect([])):
        with pytest.raises(lbm.LbmError) as ei:
            call()
        assert ei.value.status == lbm.LBM_EINVAL
