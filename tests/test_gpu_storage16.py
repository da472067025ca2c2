"""16-bit population storage (lbm_params.precision = LBM_FP16 / LBM_BF16)
against the FP64 oracle, through the C ABI.

The populations are kept as FP32 rest values m = M/36 per node (M the
zeroth moment of the set) plus 16-bit deviations dev_a = f_a - k_a m(source)
with the integer weights k_a = 36 w_a = 16, 4, 1.  The arithmetic stays
FP32, so the errors below come from rounding the deviations: a relative
2^-11 (binary16) or 2^-8 (bfloat16) of each deviation per step.  Deviations
are the velocity, flux and non-equilibrium content of a population (the
conserved scalars ride in m), so the tolerances are stated per observable,
measured against each field's magnitude (velocities against the velocity
scale U_o of Eq. (21)):

  field        binary16   bfloat16   (max error after the 2000 steps of the
  phi          3e-4       2e-3        64x128 channel; measured 9e-5-1.3e-4
  u / U_o      1e-2       3e-2        and 4.6e-4-5.3e-4 phi, 2.4e-3 and
  p            1e-2       5e-2        8.7e-3 u, 3.8e-3 and 1.9e-2 p, 2.3e-5
  T            1e-4       5e-4        and 1.1e-4 T, 3e-5-1.5e-4 and 2.1e-4
  psi          3e-4       1e-3        psi)

and the bubble centroid within 0.5 % of R (measured 5e-4 lu binary16, 8e-4
lu bfloat16 at R = 12)."""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu

FIELD = ("phi", "ux", "uy", "p", "T", "psi")
PREC = {"fp16": 1, "bf16": 2}
UNIT = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}   # half an ulp, relative
FLOOR = {"fp16": 2.0 ** -25, "bf16": 0.0}         # half the binary16 subnormal spacing
TOL_2000 = {"fp16": dict(phi=3e-4, ux=1e-2, uy=1e-2, p=1e-2, T=1e-4, psi=3e-4),
            "bf16": dict(phi=2e-3, ux=3e-2, uy=3e-2, p=5e-2, T=5e-4, psi=1e-3)}
E = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


@pytest.fixture(scope="module")
def lbm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2408_00146_gb300 import lbm as L
    L.load()
    return L


def _rows(p):
    return slice(1, p["ny"] - 1) if p["walls"] else slice(None)


def _field_errors(a, b, p, U):
    r = _rows(p)
    out = {}
    for k, name in enumerate(FIELD):
        den = U if name in ("ux", "uy") else max(np.abs(b[k, r]).max(), 1e-30)
        out[name] = np.abs(a[k, r] - b[k, r]).max() / den
    return out


def _with(p, prec):
    q = dict(p)
    q["precision"] = PREC[prec]
    return q


def _source_field(field, a, walls):
    """field at the source y - e_a of population a at every node, or at the
    node itself where y - e_a is a wall row (the population bounced back)."""
    src = np.roll(np.roll(field, E[a, 0], axis=1), E[a, 1], axis=0)
    if walls:
        ny = field.shape[0]
        if E[a, 1] == 1:
            src[1] = field[1]
        if E[a, 1] == -1:
            src[ny - 2] = field[ny - 2]
    return src


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_initial_populations_within_storage_rounding(lbm, orc, prec):
    """Each rebuilt initial population differs from the oracle's equilibrium
    by at most the rounding of its deviation (half an ulp of the format, or
    half the subnormal spacing for binary16 deviations below 2^-14), the
    rounding errors of the source node's nine deviations that its M carries,
    and FP32 rounding."""
    p = _with(si.channel_64x128(), prec)
    f = si.parity_fields(p, seed=0)
    sim = lbm.Sim(p)
    sim.init(f)
    o = orc.Oracle(p)
    o.init_fields(f)
    got = sim.populations().astype(np.float64)
    ref = o.populations()
    r = _rows(p)
    for s, k in enumerate((0, 3, 4, 5)):          # M of f, g, h, q: phi, p, T, psi
        dev = np.stack([ref[s, a] - W[a] * _source_field(f[k], a, p["walls"])
                        for a in range(9)])
        dmax = np.abs(dev[:, r]).max()
        for a in range(9):
            bound = (UNIT[prec] * (np.abs(dev[a]) + 9 * W[a] * dmax)
                     + FLOOR[prec] * (1 + 9 * W[a]) + 4e-7 * np.abs(ref[s]).max() + 1e-12)
            err = np.abs(got[s, a] - ref[s, a])
            assert np.all(err[r] <= bound[r]), (s, a, float((err[r] / bound[r]).max()))


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("noise", [False, True])
def test_channel_64x128_2000_steps(lbm, orc, prec, noise):
    p = _with(si.channel_64x128(), prec)
    f = si.parity_fields(p, seed=0) if noise else si.bubble_fields(p)
    sim = lbm.Sim(p)
    sim.init(f)
    o = orc.Oracle(p)
    o.init_fields(f)
    sim.step(2000)
    o.step(2000)
    a, b = sim.observe(), o.observe()
    Uo = b["U_o"]
    ferr = _field_errors(sim.fields(), o.fields(), p, Uo)
    for name, tol in TOL_2000[prec].items():
        assert ferr[name] <= tol, (name, ferr)
    R = p["R"]
    assert abs(a["xc"] - b["xc"]) <= 0.005 * R and abs(a["yc"] - b["yc"]) <= 0.005 * R, (a, b)
    assert abs(a["yc"] - b["yc"]) <= (2e-3 if prec == "fp16" else 5e-3), (a["yc"], b["yc"])
    assert abs(a["uy_bub"] - b["uy_bub"]) <= (5e-3 if prec == "fp16" else 2e-2) * Uo
    assert a["mass_phi"] == pytest.approx(b["mass_phi"], rel=1e-5)
    assert a["mass_psi"] == pytest.approx(b["mass_psi"], rel=1e-5)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("nx,ny,walls", [(45, 37, 1), (37, 29, 0), (4, 5, 1), (4, 4, 0),
                                         (33, 9, 1), (70, 19, 0),
                                         # streaming: partial last column and chunk, an
                                         # 8-wide last column; periodic y (rest-moment
                                         # rows wrapped), also with a partial column
                                         (80, 63, 1), (40, 21, 1), (40, 24, 0), (80, 32, 0)])
def test_ragged_and_minimal_lattices(lbm, orc, prec, nx, ny, walls):
    """Partial tiles (or a partial last column and chunk of the streaming
    kernel), the smallest lattices, both boundary modes, 30 steps.
    On the bubble-free lattices p and u are the seeded noise alone, so p is
    measured against rho_A max|u| as well as its own size."""
    p = si.scaled_channel(nx, ny)
    R = min(nx, ny) / 5.0
    p.update(walls=walls, R=R, xb=nx / 2, yb=ny / 2)
    if R < p["W"]:
        p.update(R=0.0, nu_A=0.0335, alpha_A=3.35e-3)
    p = _with(p, prec)
    f = si.parity_fields(p, seed=7)
    sim = lbm.Sim(p)
    sim.init(f)
    nfy = ny - 2 if walls else ny
    streams = nx % 8 == 0 and nx >= 32 and nfy >= 16 and (bool(walls) or nfy % 8 == 0)
    assert (lbm.lbm_batch_plan([sim])[0] > 0) == streams
    o = orc.Oracle(p)
    o.init_fields(f)
    sim.step(30)
    o.step(30)
    a, b = sim.fields(), o.fields()
    r = _rows(p)
    umax = max(np.abs(b[1:3, r]).max(), 1e-30)
    tol = 2e-4 if prec == "fp16" else 2e-3
    for k in (0, 4, 5):
        den = max(np.abs(b[k, r]).max(), 1e-30)
        assert np.abs(a[k, r] - b[k, r]).max() <= tol * den, (FIELD[k], k)
    assert np.abs(a[1:3, r] - b[1:3, r]).max() <= 3e-2 * umax
    pden = np.abs(b[3, r]).max() + p["rho_A"] * umax
    assert np.abs(a[3, r] - b[3, r]).max() <= 3e-2 * pden


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_rest_state_is_a_fixed_point(lbm, prec):
    """Uniform fields at rest with equal wall temperatures: every deviation
    is zero or the FP32 rounding of w_a M, and the state does not move."""
    p = si.scaled_channel(64, 64)
    p.update(R=0.0, nu_A=0.05, alpha_A=0.05, T_H=0.5, T_C=0.5)
    p = _with(p, prec)
    sim = lbm.Sim(p)
    sim.init(si.uniform_fields(p))
    f0, p0 = sim.fields(), sim.populations()
    sim.step(100)
    assert np.abs(sim.fields() - f0).max() <= 1e-6
    assert np.abs(sim.populations() - p0).max() <= 1e-6


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_mass_conserved_over_1000_steps(lbm, prec):
    """The rounding errors of the deviations a node pushes are folded into
    its FP32 M: sum phi and sum psi stay within FP32-level drift."""
    p = _with(si.channel_64x128(), prec)
    sim = lbm.Sim(p)
    sim.init(si.bubble_fields(p))
    m0 = sim.observe()
    sim.step(1000)
    m1 = sim.observe()
    assert m1["mass_phi"] == pytest.approx(m0["mass_phi"], rel=5e-6)
    assert m1["mass_psi"] == pytest.approx(m0["mass_psi"], rel=5e-6)


def test_graph_replay_equals_single_launches(lbm):
    p = _with(si.channel_64x128(), "fp16")
    f = si.parity_fields(p, seed=1)
    a = lbm.Sim(p)
    a.init(f)
    a.step(3)
    a.step(130)
    b = lbm.Sim(p)
    b.init(f)
    for _ in range(133):
        b.step(1)
    assert np.array_equal(a.populations(), b.populations())


def test_batch_with_mixed_precisions_equals_separate_steps(lbm):
    """One lbm_step_batch call over sims of all three storage precisions (one
    launch per precision per step) equals stepping each alone."""
    import torch
    ps = [_with(si.channel_64x128(), "fp16"), _with(si.scaled_channel(45, 37), "bf16"),
          si.channel_256x1024(0.2, 5e-4), _with(si.channel_256x1024(0.1, 1e-3), "fp16")]
    ps[1].update(R=7.0)
    fields = [si.parity_fields(p, seed=20 + i) for i, p in enumerate(ps)]
    st = torch.cuda.Stream()
    batch = [lbm.Sim(p, stream=st) for p in ps]
    alone = [lbm.Sim(p, stream=st) for p in ps]
    for s, f in zip(batch + alone, fields + fields):
        s.init(f)
    lbm.lbm_step_batch(batch, 7)
    for s in alone:
        s.step(7)
    for a, b in zip(batch, alone):
        assert np.array_equal(a.populations(), b.populations())
    assert batch[0].launches() >= 7 * 3


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_restart_from_populations(lbm, prec):
    """A checkpoint (FP32 populations) restarts a 16-bit sim: the rebuilt
    populations match the checkpoint to the format's rounding, and the run
    continues as the uninterrupted one to the same order."""
    p = _with(si.channel_64x128(), prec)
    f = si.parity_fields(p, seed=2)
    a = lbm.Sim(p)
    a.init(f)
    a.step(40)
    ck = a.populations()
    b = lbm.Sim(p)
    b.init(populations=ck)
    back = b.populations()
    r = _rows(p)
    for s in range(4):
        den = np.abs(ck[s, :, r]).max()
        assert np.abs(back[s, :, r] - ck[s, :, r]).max() <= 4 * UNIT[prec] * den
    assert b.observe()["mass_phi"] == pytest.approx(a.observe()["mass_phi"], rel=1e-6)
    a.step(40)
    b.step(40)
    Uo = a.observe()["U_o"]
    ferr = _field_errors(b.fields(), a.fields(), p, Uo)
    for name, tol in TOL_2000[prec].items():
        assert ferr[name] <= tol, (name, ferr)


def test_fp32_checkpoint_into_fp16_sim(lbm, orc):
    p32 = si.channel_64x128()
    f = si.parity_fields(p32, seed=3)
    a = lbm.Sim(p32)
    a.init(f)
    a.step(25)
    b = lbm.Sim(_with(p32, "fp16"))
    b.init(populations=a.populations())
    b.step(25)
    a.step(25)
    ferr = _field_errors(b.fields(), a.fields(), p32, a.observe()["U_o"])
    for name, tol in TOL_2000["fp16"].items():
        assert ferr[name] <= tol, (name, ferr)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_full_size_1024x4096(lbm, orc, prec):
    """Full 1024x4096 lattice (R = 96), every node, two steps."""
    p = _with(si.channel_1024x4096(), prec)
    f = si.parity_fields(p, seed=12)
    sim = lbm.Sim(p)
    sim.init(f)
    o = orc.Oracle(p)
    o.init_fields(f)
    sim.step(2)
    o.step(2)
    a, b = sim.observe(), o.observe()
    ferr = _field_errors(sim.fields(), o.fields(), p, max(np.abs(o.fields()[1:3]).max(), 1e-30))
    tol = TOL_2000[prec]
    for name in ("phi", "T", "psi"):
        assert ferr[name] <= tol[name], (name, ferr)
    assert max(ferr["ux"], ferr["uy"]) <= 5 * tol["ux"], ferr
    assert a["mass_phi"] == pytest.approx(b["mass_phi"], rel=1e-6)
    assert abs(a["yc"] - b["yc"]) < 1e-3
