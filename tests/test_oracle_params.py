"""Pins of the oracle's parameter derivation, surface-tension law, adsorption
potential and isotropic stencils against the paper's definitions.  CPU only."""
import numpy as np
import pytest

import seeded_inputs as si


def test_derived_parameters_solve_the_paper_definitions(orc):
    """U_o, nu_A, alpha_A jointly satisfy Re = U R / nu_A, Ma = U R / alpha_A
    (Eq. (8)) and U_o = (sigma0 / mu_A)(R / L)(M1 + M2) (Eq. (21)), with M1,
    M2 from Eq. (10); ratios from Eq. (9); rates from M = c_s^2 (1/w - 1/2)
    (App. B, E); Pi = lambda W^2 / (8 sigma0) and Ex = 4 s / (w W^2)
    (groups defined after Eq. (11))."""
    for p in (si.channel_64x128(), si.channel_256x1024(0.2, 5e-4), si.channel_1024x4096()):
        d = orc.derive(p)
        R, L = p["R"], p["ny"]
        assert d["M1"] == pytest.approx(p["sigma_T"] * (p["T_H"] - p["T_C"]) / p["sigma0"])
        assert d["M2"] == pytest.approx(p["sigma_TT"] * (p["T_H"] - p["T_C"]) ** 2 / p["sigma0"])
        assert d["U_o"] * R / d["nu_A"] == pytest.approx(p["Re"], rel=1e-13)
        assert d["U_o"] * R / d["alpha_A"] == pytest.approx(p["Ma"], rel=1e-13)
        assert d["U_o"] == pytest.approx(
            p["sigma0"] / d["mu_A"] * (R / L) * (d["M1"] + d["M2"]), rel=1e-13)
        assert d["rho_A"] / d["rho_B"] == pytest.approx(p["rho_ratio"])
        assert d["mu_A"] / d["mu_B"] == pytest.approx(p["mu_ratio"])
        assert d["mu_A"] == pytest.approx(d["rho_A"] * d["nu_A"])
        assert d["nu_B"] == pytest.approx(d["mu_B"] / d["rho_B"])
        assert (1 / 3) * (1 / d["omega_phi"] - 0.5) == pytest.approx(p["M_phi"])
        assert (1 / 3) * (1 / d["omega_psi"] - 0.5) == pytest.approx(p["M_psi"])
        assert d["lambda"] * p["W"] ** 2 / (8 * p["sigma0"]) == pytest.approx(p["Pi"])
        assert 4 * d["s"] / (d["w"] * p["W"] ** 2) == pytest.approx(p["Ex"])
        # reading R7: Pi = lambda W^2 / s, adsorption flux m_psi = D_psi / lambda
        assert d["lambda"] * p["W"] ** 2 / d["s"] == pytest.approx(p["Pi"])
        assert d["m_psi"] * d["lambda"] == pytest.approx(d["D_psi"])


def test_surfactant_model_parameters_of_sec6(orc):
    """Sec. 6 fixes sigma0 = 5e-3, W = 5, Ex = 0.16, Pi = 8.33: lambda =
    8 sigma0 Pi / W^2 = 0.0133; with s = 8 sigma0 both s and w are 0.04."""
    p = si.channel_64x128()
    p.update(W=5.0)
    d = orc.derive(p)
    assert d["lambda"] == pytest.approx(0.013328, rel=1e-4)
    assert d["s"] == pytest.approx(0.04) and d["w"] == pytest.approx(0.04)


def test_rejects_unstable_or_invalid_parameters(orc):
    p = si.channel_64x128()
    p.update(M_phi=-0.2)  # omega_phi outside (0, 2)
    with pytest.raises(ValueError):
        orc.derive(p)
    p = si.channel_64x128()
    p.update(nx=2)
    with pytest.raises(ValueError):
        orc.derive(p)
    p = si.channel_64x128()
    p.update(sigma_TT=0.0)  # no thermocapillary scale and no viscosity given
    with pytest.raises(ValueError):
        orc.derive(p)


def test_surface_tension_law(orc):
    """Eq. (6): sigma(T_ref, 0) = sigma0; sigma_T = d sigma/dT and
    sigma_TT = (1/2) d^2 sigma/dT^2 at T_ref (definitions below Eq. (6));
    Langmuir term d sigma/d psi = -sigma0 beta (T/T_ref)/(1 - psi); the
    dimensionless form Eq. (11) gives the same values."""
    p = si.channel_64x128()
    p.update(sigma_T=-2e-3, sigma_TT=3e-3, beta=0.2)
    s = lambda T, psi: orc.sigma_eos(p, T, psi)
    Tr, h = p["T_ref"], 1e-4
    assert s(Tr, 0.0) == pytest.approx(p["sigma0"], rel=1e-15)
    # at psi = 0 the Langmuir term vanishes: derivatives are pure temperature law
    dT1 = (s(Tr + h, 0.0) - s(Tr - h, 0.0)) / (2 * h)
    dT2 = (s(Tr + h, 0.0) - 2 * s(Tr, 0.0) + s(Tr - h, 0.0)) / h ** 2
    assert dT1 == pytest.approx(p["sigma_T"], rel=1e-6)
    assert 0.5 * dT2 == pytest.approx(p["sigma_TT"], rel=1e-5)
    for T, psi in [(0.3, 0.2), (0.9, 0.6)]:
        dpsi = (s(T, psi + h) - s(T, psi - h)) / (2 * h)
        assert dpsi == pytest.approx(-p["sigma0"] * p["beta"] * (T / Tr) / (1 - psi), rel=1e-6)
        dTn = p["T_H"] - p["T_C"]
        M1 = dTn * p["sigma_T"] / p["sigma0"]
        M2 = dTn ** 2 * p["sigma_TT"] / p["sigma0"]
        dimless = 1 + p["beta"] * (T / Tr) * np.log(1 - psi) + M1 * (T - Tr) / dTn + \
            M2 * (T - Tr) ** 2 / dTn ** 2
        assert s(T, psi) / p["sigma0"] == pytest.approx(dimless, rel=1e-14)


def test_surface_tension_clamp_keeps_log_finite(orc):
    p = si.channel_64x128()
    assert np.isfinite(orc.sigma_eos(p, 0.5, 1.0))
    assert np.isfinite(orc.sigma_eos(p, 0.5, 1.2))
    assert orc.sigma_eos(p, 0.5, -0.1) == pytest.approx(orc.sigma_eos(p, 0.5, 0.0))


def test_adsorption_potential_and_its_derivative(orc):
    """G of Eq. (5) with phi_m = 1/2, phi_o = -1/2: the adsorption term equals
    -(s/2)|grad phi|^2 of Eq. (2) on the tanh profile (|grad phi| =
    4 phi (1 - phi) / W), the bulk values G(0) = G(1) = w/8, and G' is the
    derivative of G."""
    p = si.channel_64x128()
    p.update(W=5.0)
    d = orc.derive(p)
    W = p["W"]
    for phi in (0.0, 1.0):
        assert orc.G(p, phi) == pytest.approx(d["w"] / 8, rel=1e-14)
    for phi in np.linspace(0.05, 0.95, 7):
        grad = 4 * phi * (1 - phi) / W
        expect = -0.5 * d["s"] * grad ** 2 + 0.5 * d["w"] * (phi - 0.5) ** 2
        assert orc.G(p, phi) == pytest.approx(expect, rel=1e-12)
        h = 1e-6
        num = (orc.G(p, phi + h) - orc.G(p, phi - h)) / (2 * h)
        assert orc.dG(p, phi) == pytest.approx(num, rel=1e-7, abs=1e-12)


def test_isotropic_gradient_stencil(orc):
    """Reading R6: grad X = 3 sum w_a e_a X(x + e_a) is exact on linear
    fields, second order on smooth ones, and isotropic: a plane wave's
    gradient error does not depend on its direction at leading order."""
    nx = ny = 64
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    # linear on the interior (periodic wrap spoils the seam rows only)
    gx, gy = orc.gradient_periodic(0.3 * x - 0.7 * y)
    assert np.allclose(gx[2:-2, 2:-2], 0.3, atol=1e-13)
    assert np.allclose(gy[2:-2, 2:-2], -0.7, atol=1e-13)
    errs = []
    for n in (16, 32, 64):
        yy, xx = np.mgrid[0:n, 0:n].astype(float)
        k = 2 * np.pi / n
        a = np.sin(k * xx) * np.cos(k * yy)
        gx, gy = orc.gradient_periodic(a)
        errs.append(np.abs(gx - k * np.cos(k * xx) * np.cos(k * yy)).max() / k)
    assert errs[0] / errs[1] == pytest.approx(4, rel=0.05)
    assert errs[1] / errs[2] == pytest.approx(4, rel=0.05)
    n = 64
    yy, xx = np.mgrid[0:n, 0:n].astype(float)
    k = 2 * np.pi * 4 / n
    a0 = np.sin(k * xx)                 # wavevector (k, 0)
    a1 = np.sin(k * (xx + yy) / 2)      # wavevector (k/2, k/2), |K| = k/sqrt2
    gx0, gy0 = orc.gradient_periodic(a0)
    gx1, gy1 = orc.gradient_periodic(a1)
    # magnitude reduction of the discrete derivative for |k| = k and |k| = k/sqrt2
    m0 = np.abs(gx0).max() / k
    m1 = np.hypot(gx1, gy1).max() / (k / np.sqrt(2))
    # isotropic stencil: reduction 1 - |k|^2/6 + O(k^4) regardless of direction
    assert 1 - m0 == pytest.approx(k ** 2 / 6, rel=0.1)
    assert 1 - m1 == pytest.approx((k / np.sqrt(2)) ** 2 / 6, rel=0.1)
