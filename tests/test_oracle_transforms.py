"""Pins of the oracle's moment transforms and collision against what the paper
prints (App. F) and against the definitions of raw and central moments
(App. B, Eq. (24)).  CPU only."""
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")
MOMENTS = [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2), (1, 1), (2, 1), (1, 2), (2, 2)]


def _load(name):
    return np.loadtxt(os.path.join(GOLD, name), comments="#")


def _printed_F(ux, uy):
    rows = []
    with open(os.path.join(GOLD, "F_matrix_printed.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([eval(c, {"__builtins__": {}}, {"ux": ux, "uy": uy})
                         for c in line.split(";")])
    return np.array(rows, dtype=float)


def _brute_central(f, ux, uy, ex, ey):
    """Central moments by their definition, App. B Eq. (24b)."""
    return np.array([np.sum(f * (ex - ux) ** m * (ey - uy) ** n) for m, n in MOMENTS])


def test_velocity_set_matches_P(orc):
    ex, ey = orc.velocities()
    P = _load("P_matrix.txt")
    # rows 10 and 01 of the printed P are e_x and e_y (App. F, Eq. (45))
    assert np.array_equal(P[1], ex) and np.array_equal(P[2], ey)
    # every direction appears once, with its opposite
    assert len({(a, b) for a, b in zip(ex, ey)}) == 9


def test_P_equals_printed(orc):
    assert np.array_equal(orc.matrix_P(), _load("P_matrix.txt"))


def test_Pinv_equals_printed_and_inverts(orc):
    Pinv = orc.matrix_Pinv()
    assert np.allclose(Pinv, _load("Pinv_matrix.txt"), atol=1e-15, rtol=0)
    assert np.allclose(orc.matrix_P() @ Pinv, np.eye(9), atol=1e-15)


def test_F_matches_central_moment_definition(orc):
    rng = np.random.default_rng(1)
    ex, ey = orc.velocities()
    P = orc.matrix_P()
    for _ in range(20):
        f = rng.uniform(-1, 1, 9)
        ux, uy = rng.uniform(-0.3, 0.3, 2)
        k = orc.matrix_F(ux, uy) @ (P @ f)
        assert np.allclose(k, _brute_central(f, ux, uy, ex, ey), atol=1e-14, rtol=0)


def test_F_inverse_is_F_of_minus_u(orc):
    rng = np.random.default_rng(2)
    for _ in range(20):
        ux, uy = rng.uniform(-0.5, 0.5, 2)
        assert np.allclose(orc.matrix_F(ux, uy) @ orc.matrix_F(-ux, -uy), np.eye(9),
                           atol=1e-15)


def test_printed_F_rows_and_last_row_misprint(orc):
    """Rows 00..12 of the printed F agree with the oracle; the printed last
    row breaks both the definition and F(u) F(-u) = I, the corrected one
    does not (reading R1)."""
    ux, uy = 0.13, -0.07
    Fp = _printed_F(ux, uy)
    Fo = orc.matrix_F(ux, uy)
    assert np.allclose(Fp[:8], Fo[:8], atol=1e-15)
    assert not np.allclose(Fp[8], Fo[8], atol=1e-6)
    assert not np.allclose(Fp @ _printed_F(-ux, -uy), np.eye(9), atol=1e-6)
    # only the two entries that lack the binomial factor differ, by that factor
    assert np.allclose(Fo[8, 1], 2 * Fp[8, 1]) and np.allclose(Fo[8, 2], 2 * Fp[8, 2])
    assert np.allclose(np.delete(Fo[8], [1, 2]), np.delete(Fp[8], [1, 2]))


def test_rest_equilibrium_is_d2q9_weights(orc):
    """The energy-scheme equilibrium at rest (App. D, Eq. (37)) with T = 1 is
    the standard D2Q9 weight set, which the stencils and the
    anti-bounce-back use."""
    eq = np.array([1, 0, 0, 1 / 3, 1 / 3, 0, 0, 0, 1 / 9])
    out = orc.cm_collide(np.zeros(9), 0.0, 0.0, eq, np.ones(9))
    assert np.allclose(out, orc.weights(), atol=1e-16)
    assert np.allclose(orc.weights(),
                       [4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 36, 1 / 36, 1 / 36, 1 / 36])


def test_unit_rates_return_equilibrium(orc):
    """With every rate 1 and no source the collision output carries exactly
    the equilibrium central moments (checked by the definition Eq. (24b))."""
    rng = np.random.default_rng(3)
    ex, ey = orc.velocities()
    for _ in range(10):
        pop = rng.uniform(0, 0.2, 9)
        ux, uy = rng.uniform(-0.1, 0.1, 2)
        eq = rng.uniform(-0.1, 0.1, 9)
        out = orc.cm_collide(pop, ux, uy, eq, np.ones(9))
        assert np.allclose(_brute_central(out, ux, uy, ex, ey), eq, atol=1e-15)


def test_relaxation_rule_per_moment(orc):
    """Each central moment follows k~ = k + w (k_eq - k) + (1 - w/2) s
    (App. C, Eq. (33)); with the split, the trace 20+02 and the deviator
    20-02 relax with their own rates."""
    rng = np.random.default_rng(4)
    ex, ey = orc.velocities()
    pop = rng.uniform(0, 0.2, 9)
    ux, uy = 0.05, -0.02
    eq = rng.uniform(-0.1, 0.1, 9)
    src = rng.uniform(-0.01, 0.01, 9)
    om = rng.uniform(0.5, 1.9, 9)
    k = _brute_central(pop, ux, uy, ex, ey)
    out = orc.cm_collide(pop, ux, uy, eq, om, src)
    kt = _brute_central(out, ux, uy, ex, ey)
    assert np.allclose(kt, k + om * (eq - k) + (1 - om / 2) * src, atol=1e-15)
    w2s, w2d = 1.1, 1.6
    out = orc.cm_collide(pop, ux, uy, eq, om, src, split=True, om2s=w2s, om2d=w2d)
    kt = _brute_central(out, ux, uy, ex, ey)
    t2s = (k[3] + k[4]) + w2s * ((eq[3] + eq[4]) - (k[3] + k[4])) + (1 - w2s / 2) * (src[3] + src[4])
    t2d = (k[3] - k[4]) + w2d * ((eq[3] - eq[4]) - (k[3] - k[4])) + (1 - w2d / 2) * (src[3] - src[4])
    assert np.allclose(kt[3] + kt[4], t2s, atol=1e-15)
    assert np.allclose(kt[3] - kt[4], t2d, atol=1e-15)
    keep = [0, 1, 2, 5, 6, 7, 8]
    assert np.allclose(kt[keep], (k + om * (eq - k) + (1 - om / 2) * src)[keep], atol=1e-15)


def test_initial_populations_carry_printed_equilibria(orc):
    """Populations the oracle builds from uniform fields carry the central
    moments of the printed equilibria (Eqs. (31), (37), (42) at R = 0), and
    the g equilibrium equals c_s^2 times the Maxwellian central moments of
    density rho plus (p - rho c_s^2) times the central moments of the rest
    weights: the incompressible transformation the paper builds on (App. C)."""
    import seeded_inputs as si
    ex, ey = orc.velocities()
    w = orc.weights()
    prm = si.channel_64x128()
    prm.update(nx=4, ny=4, walls=0, R=0.0, nu_A=0.1, alpha_A=0.1, sigma_TT=0.0)
    d = orc.derive(prm)
    phi, ux, uy, p, T, psi = 0.3, 0.04, -0.03, 3e-3, 0.8, 0.4
    fields = si.uniform_fields(prm, phi=phi, T=T, psi=psi, ux=ux, uy=uy, pressure=p)
    o = orc.Oracle(prm)
    o.init_fields(fields)
    pops = o.populations()[:, :, 1, 2]
    rho = d["rho_A"] + phi * (d["rho_B"] - d["rho_A"])
    cs2 = 1 / 3
    vp = p - rho * cs2
    maxw = np.array([rho, 0, 0, rho * cs2, rho * cs2, 0, 0, 0, rho * cs2 ** 2])
    wmom = _brute_central(w, ux, uy, ex, ey)
    assert np.allclose(_brute_central(pops[1], ux, uy, ex, ey), cs2 * maxw + vp * wmom,
                       atol=1e-16)
    scalar = np.array([1, 0, 0, cs2, cs2, 0, 0, 0, cs2 ** 2])
    # uniform phi: n = 0, so the sharpening flux vanishes (Eq. (26))
    assert np.allclose(_brute_central(pops[0], ux, uy, ex, ey), phi * scalar, atol=1e-16)
    assert np.allclose(_brute_central(pops[2], ux, uy, ex, ey), T * scalar, atol=1e-16)
    assert np.allclose(_brute_central(pops[3], ux, uy, ex, ey), psi * scalar, atol=1e-16)
    # macroscopic fields read back from those populations (Eqs. (28), (34),
    # (39), (44)); no force acts on a uniform state
    F = o.fields()
    assert np.allclose(F[:, 2, 1], [phi, ux, uy, p, T, psi], atol=1e-16)


def test_mass_preserved_by_collision(orc):
    """Zeroth moment kept by the f, h, q collisions (equilibrium k00 = the
    conserved scalar, App. B, D, E)."""
    rng = np.random.default_rng(5)
    for _ in range(10):
        pop = rng.uniform(0, 0.2, 9)
        phi = pop.sum()
        ux, uy = rng.uniform(-0.1, 0.1, 2)
        eq = np.array([phi, 0.01, -0.02, phi / 3, phi / 3, 0, 0, 0, phi / 9])
        om = np.ones(9)
        om[1] = om[2] = 1.3
        out = orc.cm_collide(pop, ux, uy, eq, om)
        assert out.sum() == pytest.approx(phi, rel=1e-14, abs=1e-15)
