"""Pins of the oracle's two-fluid property handling: the interpolation of
density, viscosity and thermal diffusivity across the phases (Eq. (17),
reading R2), the clamp of phi in that interpolation (reading R14), the
buoyancy force of Sec. 5.3, and the wall ghosts of psi and T in the surface
tension gradient (readings R10, R13).

Each pin compares the oracle with a closed form of the continuum problem in a
layered (one-dimensional) geometry.  Beside each pin, a test plants the
mistake it is meant to catch in a copy of the oracle (compiled on the CPU by
oracle.variant; the oracle's source is untouched) and checks that the same
comparison then fails.  CPU only."""
import numpy as np
import pytest

import seeded_inputs as si

# Planted mistakes: (text of lbm_oracle.c, replacement).
MUTANTS = {
    # rho interpolated from the wrong end (the printed form of Eq. (17))
    "swap_rho": [("return s->d.rho_A + phi_prop(phi) * (s->d.rho_B - s->d.rho_A);",
                  "return s->d.rho_B + phi_prop(phi) * (s->d.rho_A - s->d.rho_B);")],
    "swap_mu": [("return s->d.mu_A + phi_prop(phi) * (s->d.mu_B - s->d.mu_A);",
                 "return s->d.mu_B + phi_prop(phi) * (s->d.mu_A - s->d.mu_B);")],
    "swap_alpha": [("return s->d.alpha_A + phi_prop(phi) * (s->d.alpha_B - s->d.alpha_A);",
                    "return s->d.alpha_B + phi_prop(phi) * (s->d.alpha_A - s->d.alpha_B);")],
    # one diffusivity for both phases
    "uniform_alpha": [("return s->d.alpha_A + phi_prop(phi) * (s->d.alpha_B - s->d.alpha_A);",
                       "return s->d.alpha_A;")],
    # phi not clamped in the property interpolation (reading R14 dropped)
    "no_clamp": [("return phi < 0.0 ? 0.0 : (phi > 1.0 ? 1.0 : phi);", "return phi;")],
    # relaxation rate from the dynamic instead of the kinematic viscosity
    "nu_is_mu": [("double nu = mu_of(s, phi) / rho;", "double nu = mu_of(s, phi);")],
    # velocity without the half-force term of Eq. (34)
    "full_force": [("double ux = s->jx[i] / (rho * CS2) + 0.5 * Ftx / rho;",
                    "double ux = s->jx[i] / (rho * CS2) + Ftx / rho;")],
    # buoyancy with the wrong sign, or with rho instead of rho - rho_A
    "buoy_sign": [("- (rho - s->d.rho_A) * s->p.gravity", "+ (rho - s->d.rho_A) * s->p.gravity")],
    "buoy_rho": [("- (rho - s->d.rho_A) * s->p.gravity", "- rho * s->p.gravity")],
    # even instead of odd stencil ghosts at Dirichlet walls
    "psi_even": [("if (s->p.psi_bc == 1 && side < 0) return 2.0 * s->p.psi_L - v;",
                  "if (0) return 2.0 * s->p.psi_L - v;")],
    "T_even": [("if (side < 0) return 2.0 * s->p.T_H - v;", "if (side < 0) return v;")],
}


def _library(orc, tag):
    return None if tag is None else orc.variant(tag, MUTANTS[tag])


def _quiet(p, **kw):
    """No surface tension, thermocapillarity or surfactant coupling; uniform
    temperature; viscosity and diffusivity given directly."""
    p = dict(p)
    p.update(sigma0=0.0, sigma_T=0.0, sigma_TT=0.0, beta=0.0, Pi=0.0, Ex=0.0, nu_A=0.1,
             alpha_A=0.1, T_H=0.5, T_C=0.5, R=0.0)
    p.update(kw)
    return p


def _steady(o, ny, field, every=1000, tol=1e-7, max_steps=200000):
    """Steps until one field's column changes by less than tol of its size
    over `every` steps."""
    prev = None
    while o.t < max_steps:
        o.step(every)
        v = o.fields()[field, 1:ny - 1, 1]
        if prev is not None and np.abs(v - prev).max() <= tol * np.abs(v).max():
            break
        prev = v
    return o.fields()


def _integral_profile(y_nodes, coef, lo, hi):
    """I(y) = int_lo^y ds / coef(s), coef linear between the node values and
    constant from the last node to the wall planes lo, hi; returns
    (fine grid, I on it)."""
    ys = np.concatenate([[lo], y_nodes, [hi]])
    cs = np.concatenate([[coef[0]], coef, [coef[-1]]])
    yf = np.linspace(lo, hi, 40001)
    cf = np.interp(yf, ys, cs)

    def cum(v):
        return np.concatenate([[0.0], np.cumsum(0.5 * (v[1:] + v[:-1]) * np.diff(yf))])
    return yf, cum(1.0 / cf), cum(yf / cf)


def _phase_clamped(phi):
    return np.clip(phi, 0.0, 1.0)


# ---------------------------------------------------------------- density

def _layer_acceleration(orc, tag=None, overshoot=1.0):
    """Uniform body force G on a periodic two-layer fluid at rest: far from
    the interfaces each layer accelerates freely, rho du/dt = G, and the
    velocity of Eq. (34) (with its half-force term) is u = G (t + 1/2) / rho
    after t steps.  Returns the relative errors in the light (B) and heavy (A)
    layer."""
    G, ny, t = 1e-6, 256, 100
    p = _quiet(si.channel_64x128(), nx=4, ny=ny, walls=0, Fext_x=G, rho_ratio=10.0,
               mu_ratio=10.0, M_phi=1e-4)
    f = si.slab_fields(p, 64.0, 192.0)
    f[0] *= overshoot
    d = orc.derive(p)
    o = orc.Oracle(p, _library(orc, tag))
    o.init_fields(f)
    o.step(t)
    F = o.fields()
    eB = F[1, 128, 0] / (G * (t + 0.5) / d["rho_B"]) - 1.0
    eA = F[1, 0, 0] / (G * (t + 0.5) / d["rho_A"]) - 1.0
    return abs(eB), abs(eA)


def test_layers_accelerate_with_their_own_density(orc):
    """rho(phi) of Eq. (17) (reading R2) enters the velocity u = j/(rho c_s^2)
    + F_t/(2 rho): each bulk phase takes its own density, and a phase field
    that overshoots 1 (here 1.05, held by a tiny mobility) still takes rho_B
    (reading R14)."""
    for ov in (1.0, 1.05):
        eB, eA = _layer_acceleration(orc, overshoot=ov)
        assert eB < 1e-9 and eA < 1e-9, (ov, eB, eA)


@pytest.mark.parametrize("tag,overshoot", [("swap_rho", 1.0), ("full_force", 1.0),
                                           ("no_clamp", 1.05)])
def test_layer_acceleration_catches(orc, tag, overshoot):
    assert max(_layer_acceleration(orc, tag, overshoot)) > 0.05


# ---------------------------------------------------------------- viscosity

def _layered_poiseuille(orc, tag=None, W=4.0, mu_ratio=10.0, rho_ratio=1.0, max_steps=200000):
    """Body-force-driven flow through a channel whose middle third is phase B
    (flat tanh interfaces parallel to the walls).  The steady Stokes solution
    for a viscosity mu(y) is u(y) = -G int_{1/2}^y (s - y0)/mu(s) ds with the
    stress-free plane y0 fixed by u = 0 on both wall planes (textbook); mu(y)
    is Eq. (17) (R2) of the oracle's own phase field.  Returns the
    maximum error relative to the peak velocity."""
    G, nu = 1e-6, 1.0
    ny = int(12 * W) + 2
    p = _quiet(si.channel_64x128(), nx=4, ny=ny, nu_A=nu, Fext_x=G, W=W, mu_ratio=mu_ratio,
               rho_ratio=rho_ratio)
    h = ny - 2
    f = si.slab_fields(p, 0.5 + h / 3.0, 0.5 + 2.0 * h / 3.0)
    f[:, 0] = 0.0
    f[:, -1] = 0.0
    d = orc.derive(p)
    o = orc.Oracle(p, _library(orc, tag))
    o.init_fields(f)
    F = _steady(o, ny, 1, max_steps=max_steps)
    y = np.arange(1, ny - 1, dtype=float)
    mu = d["mu_A"] + _phase_clamped(F[0, 1:ny - 1, 1]) * (d["mu_B"] - d["mu_A"])
    yf, I0, I1 = _integral_profile(y, mu, 0.5, ny - 1.5)
    y0 = I1[-1] / I0[-1]
    ua = np.interp(y, yf, -G * (I1 - y0 * I0))
    u = F[1, 1:ny - 1, 1]
    assert np.abs(F[2]).max() < 1e-6 * np.abs(u).max()   # flow stays parallel
    return np.abs(u - ua).max() / np.abs(ua).max()


def test_layered_poiseuille_viscosity_ratio(orc):
    """Viscosity ratio 10 at equal densities: the velocity follows the
    piecewise-parabolic Stokes profile of mu(y) to 1 % (the residual is the
    lattice resolution of the W = 4 interface)."""
    assert _layered_poiseuille(orc) < 0.01


def test_layered_poiseuille_viscosity_catches(orc):
    assert _layered_poiseuille(orc, "swap_mu", max_steps=6000) > 0.5


def test_layered_poiseuille_density_ratio_converges(orc):
    """Viscosity and density ratio 10 together.  The pressure-based g scheme
    streams rho c_s^2 u; its extra viscous term nu u grad^2 rho is cancelled
    by the F_p sources of Eq. (32) only up to the lattice resolution of the
    interface, so the profile misses the Stokes solution by a few percent at
    W = 4 and converges at second order in the interface width (error ratio
    (4/6)^2 = 0.44 from W = 4 to W = 6)."""
    e4 = _layered_poiseuille(orc, W=4.0, rho_ratio=10.0)
    e6 = _layered_poiseuille(orc, W=6.0, rho_ratio=10.0)
    assert e4 < 0.07
    assert 0.35 < e6 / e4 < 0.55, (e4, e6)


def test_layered_poiseuille_density_ratio_catches(orc):
    """omega from mu instead of nu = mu/rho: the stress is off by rho."""
    assert _layered_poiseuille(orc, "nu_is_mu", rho_ratio=10.0) > 0.5


# ---------------------------------------------------------------- diffusivity

def _layered_conduction(orc, tag=None):
    """Steady conduction between the Dirichlet walls (T_H at y = 1/2, T_C at
    y = ny - 3/2) through a layered medium: the flux alpha dT/dy is uniform,
    so T(y) = T_H + (T_C - T_H) I(y)/I(ny - 3/2), I(y) = int dy/alpha(y)
    (textbook), alpha(y) from Eq. (17) (R2, R14); thermal diffusivity ratio
    alpha_A/alpha_B = 4, i.e. conductivity ratio k_A/k_B = 4 (Eq. (9)).
    Returns the maximum error relative to T_H - T_C."""
    ny = 50
    p = _quiet(si.channel_64x128(), nx=4, ny=ny, T_H=1.0, T_C=0.0, alpha_A=0.2,
               alpha_ratio=4.0)
    h = ny - 2
    f = si.slab_fields(p, 0.5 + h / 3.0, 0.5 + 2.0 * h / 3.0, T=0.5)
    f[4] = si.linear_wall_temperature(p)
    f[:, 0] = 0.0
    f[:, -1] = 0.0
    d = orc.derive(p)
    o = orc.Oracle(p, _library(orc, tag))
    o.init_fields(f)
    F = _steady(o, ny, 4, tol=1e-9)
    y = np.arange(1, ny - 1, dtype=float)
    al = d["alpha_A"] + _phase_clamped(F[0, 1:ny - 1, 1]) * (d["alpha_B"] - d["alpha_A"])
    yf, I0, _ = _integral_profile(y, al, 0.5, ny - 1.5)
    Ta = 1.0 - np.interp(y, yf, I0) / I0[-1]
    return np.abs(F[4, 1:ny - 1, 1] - Ta).max()


def test_layered_conduction_diffusivity_ratio(orc):
    assert _layered_conduction(orc) < 2e-3


@pytest.mark.parametrize("tag", ["swap_alpha", "uniform_alpha"])
def test_layered_conduction_catches(orc, tag):
    assert _layered_conduction(orc, tag) > 0.02


# ---------------------------------------------------------------- buoyancy

def _hydrostatic_column(orc, tag=None):
    """A layer of the light phase B between two layers of A in a walled
    column, gravity g, buoyancy -(rho - rho_A) g (Sec. 5.3), no surface
    tension.  At rest grad p = F_t, so p(y) = p0 - g int (rho(y) - rho_A) dy
    (hydrostatics): the pressure rises by g (rho_A - rho_B) h across the
    layer and is flat in A.  Returns the maximum error relative to the
    pressure jump and the largest velocity."""
    g, ny = 1e-5, 66
    p = _quiet(si.channel_64x128(), nx=4, ny=ny, gravity=g, rho_ratio=10.0, mu_ratio=1.0,
               nu_A=0.3)
    f = si.slab_fields(p, 22.0, 44.0)
    f[:, 0] = 0.0
    f[:, -1] = 0.0
    d = orc.derive(p)
    o = orc.Oracle(p, _library(orc, tag))
    o.init_fields(f)
    o.step(8000)
    F = o.fields()
    phi, pr = F[0, 1:ny - 1, 1], F[3, 1:ny - 1, 1]
    rho = d["rho_A"] + _phase_clamped(phi) * (d["rho_B"] - d["rho_A"])
    Fy = -(rho - d["rho_A"]) * g
    pe = np.concatenate([[0.0], np.cumsum(0.5 * (Fy[1:] + Fy[:-1]))])
    pe += (pr - pe).mean()
    jump = np.abs(pe - pe.mean()).max()
    return np.abs(pr - pe).max() / jump, np.abs(F[1:3]).max()


def test_hydrostatic_two_layer_column(orc):
    err, umax = _hydrostatic_column(orc)
    assert err < 5e-3
    assert umax < 1e-7


@pytest.mark.parametrize("tag", ["swap_rho", "buoy_sign", "buoy_rho"])
def test_hydrostatic_two_layer_column_catches(orc, tag):
    assert _hydrostatic_column(orc, tag)[0] > 0.5


# ---------------------------------------------------------------- wall ghosts

def _marangoni_at_wall(orc, kind, tag=None):
    """Surface-tension gradient at the first fluid rows.  A flat interface
    normal to the walls (phi varies along x only) meets a temperature or
    surfactant profile that is linear between its Dirichlet wall values.  At
    t = 0 the fluid is at rest, so the velocity of Eq. (34) is F_t/(2 rho)
    and, with n = (+-1, 0), its y part is delta_s dsigma/dy: the Marangoni
    stress along the interface (Eq. (15)).  A Dirichlet value at the wall plane
    with a linear profile means the profile continues linearly past the wall,
    so dsigma/dy at the first row must be the smooth continuation of the
    interior one:
      T (linear law, sigma_T):            dsigma/dy uniform up to the wall;
      psi (Gibbs term, T = T_ref):        dsigma/dy ~ 1/(1 - psi(y)) (Eq. (6)).
    Returns the largest deviation of u_y(row)/u_y(row 5) from that ratio."""
    nx, ny = 32, 34
    p = _quiet(si.channel_64x128(), nx=nx, ny=ny, sigma0=5e-3, nu_A=0.3)
    if kind == "psi":
        p.update(beta=0.2, psi_bc=1, psi_L=0.4, psi_R=0.1)
    else:
        p.update(sigma_T=-1e-3, T_H=1.0, T_C=0.0)
    x = np.arange(nx, dtype=float)[None, :] * np.ones((ny, 1))
    f = np.zeros((6, ny, nx))
    f[0] = 0.5 * (np.tanh(2.0 * (x - 8.0) / p["W"]) - np.tanh(2.0 * (x - 24.0) / p["W"]))
    f[4] = si.linear_wall_temperature(p)
    f[5] = si.initial_psi(p)
    f[:, 0] = 0.0
    f[:, -1] = 0.0
    o = orc.Oracle(p, _library(orc, tag))
    o.init_fields(f)
    F = o.fields()
    uy = F[2, 1:ny - 1, 8]
    ref = F[2, 5, 8]
    if kind == "psi":
        psi = F[5, 1:ny - 1, 8]
        expect = (1.0 - F[5, 5, 8]) / (1.0 - psi)
    else:
        expect = np.ones(ny - 2)
    return np.abs(uy / ref - expect).max()


@pytest.mark.parametrize("kind", ["T", "psi"])
def test_marangoni_stress_continuous_to_dirichlet_walls(orc, kind):
    """Readings R10 (T odd about T_w) and R13 (psi odd about psi_w when held
    at psi_L / psi_R)."""
    assert _marangoni_at_wall(orc, kind) < 1e-4


@pytest.mark.parametrize("kind,tag", [("T", "T_even"), ("psi", "psi_even")])
def test_marangoni_stress_at_walls_catches(orc, kind, tag):
    assert _marangoni_at_wall(orc, kind, tag) > 0.2
