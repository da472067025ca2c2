"""The density-ratio limit of the two-fluid scheme as read (App. C,
Eqs. (31)-(34)): a pin of the oracle's behaviour on the cleanest moving
two-phase problem, a bubble carried by a uniform flow.

Without surface tension, forces or gravity, a bubble of light fluid in a
periodic box with uniform initial velocity u0 and uniform pressure is an
exact solution of the continuum equations: u stays u0 everywhere.  The g
scheme carries the momentum rho c_s^2 u (its first moment, Eq. (34)) while
rho follows the phase field of the separate f scheme (Eq. (17)); the
pressure source Gamma = F_p . u and the second-order sources of Eq. (32),
with F_p = -grad(p - rho c_s^2) on the isotropic stencil of Sec. 3, cancel
the mismatch of the two transports only up to the stencil's truncation
error.  The oracle shows exactly that:

* the velocity error is linear in u0 and falls at second order in the
  interface width W (a discretisation error, not a mistake in a term);
* it grows with rho_A/rho_B, because u = J/(rho c_s^2) divides the momentum
  error by the light phase's density;
* from a ratio of about 50 the scheme diverges within ~100 steps, and at
  100 within ~50 -- the paper's ratio of 1000 is out of reach of the scheme
  as printed.

Three other readings of App. C are planted in copies of the oracle and do
worse: F_p also in the momentum source and the velocity of Eq. (34), the
second-order sources without their F_p terms, and no pressure source at all.
If a later reading makes the oracle stable at high density ratios, the last
two tests here fail and have to be revised with it.  CPU only."""
import numpy as np
import pytest

import seeded_inputs as si

READINGS = {
    "fp_in_momentum": [
        ("    sg[1] = CS2 * Ftx - ux * G;\n    sg[2] = CS2 * Fty - uy * G;",
         "    sg[1] = CS2 * (Ftx + Fpx) - ux * G;\n    sg[2] = CS2 * (Fty + Fpy) - uy * G;"),
        ("            double ux = s->jx[i] / (rho * CS2) + 0.5 * Ftx / rho;\n"
         "            double uy = s->jy[i] / (rho * CS2) + 0.5 * Fty / rho;",
         "            double ux = s->jx[i] / (rho * CS2) + 0.5 * (Ftx - pgx) / rho;\n"
         "            double uy = s->jy[i] / (rho * CS2) + 0.5 * (Fty - pgy) / rho;"),
    ],
    "no_fp_second_order": [
        ("    sg[3] = 2.0 * CS2 * Fpx * ux + (ux * ux + CS2) * G;\n"
         "    sg[4] = 2.0 * CS2 * Fpy * uy + (uy * uy + CS2) * G;\n"
         "    sg[5] = CS2 * (Fpx * uy + Fpy * ux) + ux * uy * G;",
         "    sg[3] = 0.0;\n    sg[4] = 0.0;\n    sg[5] = 0.0;"),
    ],
    "no_pressure_source": [
        ("    double G = Fpx * ux + Fpy * uy;\n    sg[0] = G;",
         "    double G = 0.0 * (Fpx * ux + Fpy * uy);\n    sg[0] = G;"),
    ],
}


def _advected(orc, ratio, u0=0.01, W=4.0, n=64, R=12.0, checkpoints=(100,), library=None):
    """Max |u - u0| / u0 at each checkpoint step (inf once non-finite or
    above 100 u0)."""
    p = si.channel_64x128()
    p.update(nx=n, ny=n, walls=0, R=R, xb=n / 2.0, yb=n / 2.0, W=W, rho_ratio=float(ratio),
             mu_ratio=1.0, alpha_ratio=1.0, sigma0=0.0, sigma_T=0.0, sigma_TT=0.0, beta=0.0,
             nu_A=0.1, alpha_A=0.05)
    f = si.bubble_fields(p)
    f[1] = u0
    o = orc.Oracle(p, library=library)
    o.init_fields(f)
    out = []
    for t in checkpoints:
        e = np.inf
        try:
            o.step(t - o.t)
            fl = o.fields()
            e = float(np.hypot(fl[1] - u0, fl[2]).max()) / u0
        except RuntimeError:
            pass
        if not np.isfinite(e) or e > 100.0:
            out += [np.inf] * (len(checkpoints) - len(out))
            break
        out.append(e)
    o.close()
    return out


def test_error_is_second_order_in_the_interface_width(orc):
    (e4,) = _advected(orc, 10, W=4.0, n=96, R=24.0, checkpoints=(1,))
    (e8,) = _advected(orc, 10, W=8.0, n=96, R=24.0, checkpoints=(1,))
    assert 0.03 < e4 < 0.3
    assert 3.0 < e4 / e8 < 5.0          # (8/4)^2 = 4


def test_error_is_linear_in_the_speed(orc):
    a = _advected(orc, 10, u0=0.005, checkpoints=(5, 20))
    b = _advected(orc, 10, u0=0.01, checkpoints=(5, 20))
    assert np.allclose(a, b, rtol=0.05)


def test_error_grows_with_the_density_ratio(orc):
    steps = tuple(range(20, 301, 20))
    e10 = max(_advected(orc, 10, checkpoints=steps))
    e20 = max(_advected(orc, 20, checkpoints=steps))
    e30 = max(_advected(orc, 30, checkpoints=steps))
    assert e10 < 0.3 and 1.5 * e10 < e20 < 1.0 and e30 > 2.0 * e20


def test_scheme_as_read_diverges_from_density_ratio_50(orc):
    assert _advected(orc, 50, checkpoints=(300,)) == [np.inf]
    assert _advected(orc, 100, checkpoints=(100,)) == [np.inf]
    assert _advected(orc, 1000, checkpoints=(30,)) == [np.inf]


@pytest.mark.parametrize("reading", sorted(READINGS))
def test_other_readings_do_worse(orc, reading):
    lib = orc.variant("dr_" + reading, READINGS[reading])
    steps = tuple(range(20, 201, 20))
    printed = max(_advected(orc, 10, checkpoints=steps))
    other = max(_advected(orc, 10, checkpoints=steps, library=lib))
    assert other > 2.0 * printed
    assert _advected(orc, 100, checkpoints=(100,), library=lib) == [np.inf]
