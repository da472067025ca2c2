"""Surfactant wall conditions on the GPU (psi_bc, Sec. 2 and Sec. 6): psi
held at psi_L / psi_R on the wall planes (1) or set only as the initial
linear profile with zero-flux walls (2).  Parity with the FP64 oracle on the
streaming kernel (walls, nx a multiple of 32), the tile kernel and 16-bit
storage; the analytic initial state; and the steady Dirichlet profile."""
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


def _case(nx, psi_bc, precision=0):
    """A bubble next to the walls (so that its stencils reach the wall
    ghosts), a strong Gibbs term (beta = 0.3) so that sigma depends on psi,
    and psi_L = 0.4, psi_R = 0.1."""
    p = si.scaled_channel(nx, 48)
    p.update(R=6.0, yb=9.0, beta=0.3, psi_L=0.4, psi_R=0.1, psi_bc=psi_bc,
             precision=precision)
    return p


@pytest.mark.parametrize("psi_bc", [1, 2])
@pytest.mark.parametrize("nx,precision", [(64, 0), (40, 0), (64, 1)])
def test_psi_walls_match_oracle(lbm, orc, psi_bc, nx, precision):
    p = _case(nx, psi_bc, precision)
    f = si.parity_fields(p, seed=3)
    sim = lbm.Sim(p)
    sim.init(f)
    o = orc.Oracle(p)
    o.init_fields(f)
    for n in (1, 40):
        sim.step(n)
        o.step(n)
        a, b = sim.fields(), o.fields()
        r = slice(1, -1)
        umax = max(np.abs(b[1:3, r]).max(), 1e-30)
        if precision == 0:
            # FP32 storage: every field within 1e-4 of its own magnitude
            for k in range(6):
                den = umax if k in (1, 2) else max(np.abs(b[k, r]).max(), 1e-30)
                assert np.abs(a[k, r] - b[k, r]).max() <= 1e-4 * den, (n, k)
        else:
            # binary16 deviations: the tolerances of the 16-bit parity tests
            for k in (0, 4, 5):
                den = max(np.abs(b[k, r]).max(), 1e-30)
                assert np.abs(a[k, r] - b[k, r]).max() <= 2e-4 * den, (n, k)
            assert np.abs(a[1:3, r] - b[1:3, r]).max() <= 3e-2 * umax, n
            pden = np.abs(b[3, r]).max() + p["rho_A"] * umax
            assert np.abs(a[3, r] - b[3, r]).max() <= 3e-2 * pden, n
    ob, oo = sim.observe(), o.observe()
    assert ob["mass_psi"] == pytest.approx(oo["mass_psi"], rel=1e-5)


@pytest.mark.parametrize("psi_bc", [1, 2])
def test_analytic_initial_psi_profile(lbm, psi_bc):
    p = _case(64, psi_bc)
    sim = lbm.Sim(p)
    sim.init()
    psi = sim.fields()[5, 1:-1]
    ref = si.bubble_fields(p)[5, 1:-1]
    assert np.abs(psi - ref).max() < 2e-6
    assert psi[0, 0] == pytest.approx(0.4 - 0.3 * 0.5 / 46, abs=2e-6)


@pytest.mark.parametrize("nx", [64, 40])
def test_steady_dirichlet_psi_profile(lbm, nx):
    """No interface, u = 0: the q scheme relaxes to psi linear between
    psi_L on the y = 1/2 plane and psi_R on y = ny - 3/2; with zero-flux
    walls the same initial profile keeps its sum and flattens to its mean."""
    base = dict(si.channel_64x128(), nx=nx, ny=34, R=0.0, sigma_T=0.0, sigma_TT=0.0, beta=0.0,
                Pi=0.0, Ex=0.0, nu_A=0.1, alpha_A=0.1, M_psi=0.3, T_H=0.5, T_C=0.5,
                psi_L=0.4, psi_R=0.1)
    xi = np.arange(1, 33) - 0.5
    p = dict(base, psi_bc=1)
    sim = lbm.Sim(p)
    sim.init(si.uniform_fields(p, psi=0.0))
    sim.step(8000)
    psi = sim.fields()[5, 1:33]
    assert np.abs(psi - (0.4 - 0.3 * xi / 32.0)[:, None]).max() < 2e-5
    p = dict(base, psi_bc=2)
    sim = lbm.Sim(p)
    sim.init(si.bubble_fields(p))
    m0 = sim.observe()["mass_psi"]
    sim.step(8000)
    assert sim.observe()["mass_psi"] == pytest.approx(m0, rel=2e-6)
    assert np.abs(sim.fields()[5, 1:33] - 0.25).max() < 2e-5


def test_bad_psi_parameters_rejected(lbm):
    for bad in (dict(psi_bc=3), dict(psi_bc=-1), dict(psi_bc=1, psi_L=1.0),
                dict(psi_bc=1, psi_R=-0.1)):
        p = dict(_case(64, 1), **bad)
        with pytest.raises(lbm.LbmError):
            lbm.Sim(p)
