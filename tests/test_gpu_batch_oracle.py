"""One lbm_step_batch over an uneven mix of simulations, every member checked
against the FP64 oracle (not against itself): lattices of different sizes
(partial last columns, a partial last chunk, periodic lattices at FP32 and
binary16 storage), both wall modes, FP32 with binary16 and bfloat16 storage,
streaming and tile kernels, and different Gibbs elasticity, quadratic
sensitivity and Marangoni number.

Tolerances: FP32 members as the FP32 parity tests (fields within 1e-4 of each
field's magnitude, velocities of U_o; centroid within 1e-3 lattice units;
masses 1e-5); 16-bit members as the per-observable table of the 16-bit
storage tests (centroid within 0.5 % of R)."""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu

FIELD = ("phi", "ux", "uy", "p", "T", "psi")
TOL16 = {1: dict(phi=3e-4, ux=1e-2, uy=1e-2, p=1e-2, T=1e-4, psi=3e-4),
         2: dict(phi=2e-3, ux=3e-2, uy=3e-2, p=5e-2, T=5e-4, psi=1e-3)}
STEPS = 300


@pytest.fixture(scope="module")
def lbm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2408_00146_gb300 import lbm as L
    L.load()
    return L


def _member(nx, ny, walls, precision, beta, sigma_TT, Ma, R):
    p = si.scaled_channel(nx, ny)
    p.update(walls=walls, precision=precision, beta=beta, sigma_TT=sigma_TT, Ma=Ma, R=R)
    if not walls:
        # no thermal walls: a linear law along y drives the bubble instead
        p.update(sigma_TT=0.0, sigma_T=-2e-4, nu_A=0.05, alpha_A=0.02)
    return p


MIX = [
    # FP32, streaming: partial last column (80 = 2.5 x 32), partial last chunk (nfy = 61)
    _member(80, 63, 1, 0, 0.05, 5e-4, 8.0, 8.0),
    # FP32, streaming, periodic y (48 rows = 6 whole chunks)
    _member(64, 48, 0, 0, 0.2, 0.0, 20.0, 7.0),
    # FP32, tile kernel (nx not a multiple of 4)
    _member(45, 40, 1, 0, 0.1, 1e-3, 10.0, 6.0),
    # binary16, streaming, partial last column (48 = 32 + 16)
    _member(48, 96, 1, 1, 0.15, 2e-3, 30.0, 7.0),
    # bfloat16, streaming
    _member(64, 80, 1, 2, 0.25, 1e-3, 15.0, 8.0),
    # binary16, tile kernel (nx not a multiple of 8)
    _member(36, 64, 1, 1, 0.1, 4e-3, 45.0, 6.0),
    # binary16, streaming, periodic y (rest-moment rows wrapped)
    _member(48, 40, 0, 1, 0.1, 0.0, 12.0, 6.0),
]


def _rows(p):
    return slice(1, p["ny"] - 1) if p["walls"] else slice(None)


@pytest.mark.parametrize("tile_w", [None, 64])
def test_uneven_batch_matches_oracle(lbm, orc, tile_w):
    """The model's plan (32 x 8 tiles), and the 64 x 4 tile shape pinned for
    the FP32 members."""
    import torch
    st = torch.cuda.Stream()
    fields = [si.parity_fields(p, seed=60 + i) for i, p in enumerate(MIX)]
    sims = [lbm.Sim(p, stream=st) for p in MIX]
    for s, f in zip(sims, fields):
        s.init(f)
    plan = lbm.lbm_batch_plan(sims)
    assert plan[2] == 0 and plan[5] == 0                      # tile-kernel members
    assert all(plan[i] >= 4 for i in (0, 1, 3, 4, 6))         # streaming members
    if tile_w:
        # FP32 members in the wide shape (16-bit storage has 32 x 8 only)
        widths = [tile_w if p["precision"] == 0 else 32 for p in MIX]
        lbm.lbm_pin_batch_plan(sims, widths, [5] * len(MIX))
        assert all(lbm.lbm_batch_tiles(sims)[i] == (64, 4) for i in (0, 1))
        assert all(lbm.lbm_batch_tiles(sims)[i] == (32, 8) for i in (3, 4, 6))
    lbm.lbm_step_batch(sims, STEPS)
    for i, (p, f, sim) in enumerate(zip(MIX, fields, sims)):
        o = orc.Oracle(p)
        o.init_fields(f)
        o.step(STEPS)
        a, b = sim.observe(), o.observe()
        assert a["t"] == STEPS
        got, ref = sim.fields(), o.fields()
        r = _rows(p)
        Uo = b["U_o"]
        err = {}
        for k, name in enumerate(FIELD):
            den = Uo if name in ("ux", "uy") else max(np.abs(ref[k, r]).max(), 1e-30)
            err[name] = np.abs(got[k, r] - ref[k, r]).max() / den
        if p["precision"] == 0:
            assert max(err.values()) <= 1e-4, (i, err)
            assert abs(a["xc"] - b["xc"]) <= 1e-3 and abs(a["yc"] - b["yc"]) <= 1e-3, (i, a, b)
        else:
            for name, tol in TOL16[p["precision"]].items():
                assert err[name] <= tol, (i, name, err)
            R = p["R"]
            assert abs(a["xc"] - b["xc"]) <= 0.005 * R and abs(a["yc"] - b["yc"]) <= 0.005 * R
        assert a["mass_phi"] == pytest.approx(b["mass_phi"], rel=1e-5), i
        assert a["mass_psi"] == pytest.approx(b["mass_psi"], rel=1e-5), i
        o.close()
    for s in sims:
        s.close()
