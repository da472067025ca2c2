"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module holds the problem configurations (plain parameter dictionaries,
named after the workloads they describe) and generators of initial
macroscopic fields.  It computes no step of the lattice Boltzmann method: it
only lays out initial shapes (a circular bubble with the hyperbolic-tangent
interface profile of Sec. 3, a planar interface, a linear wall-to-wall
temperature, seeded noise) from which each side builds its own populations.

Field arrays are float64 of shape [6, ny, nx] in the order
phi, u_x, u_y, p, T, psi; node (x, y) sits at [:, y, x].  With walls, rows
0 and ny-1 are solid and their values are ignored.
"""
from __future__ import annotations

import copy

import numpy as np

FIELD_NAMES = ("phi", "ux", "uy", "p", "T", "psi")

# Parameter names, in the order of the C structs of both libraries.
PARAM_NAMES = (
    "nx", "ny", "walls", "R", "xb", "yb", "W", "M_phi", "rho_A", "rho_ratio",
    "mu_ratio", "alpha_ratio", "Re", "Ma", "sigma0", "sigma_T", "sigma_TT",
    "T_ref", "T_H", "T_C", "beta", "Pi", "Ex", "M_psi", "psi0", "Fext_x",
    "Fext_y", "gravity", "nu_A", "alpha_A", "psi_L", "psi_R", "psi_bc",
)

# Bubble in a periodic-x channel with a hot wall at y=0 and a cold wall at
# y=ny-1: 64x128, R=12 at (32, 40), W=4, density ratio 10, viscosity ratio 1,
# self-rewetting quadratic law sigma_TT=1e-3 (sigma_T=0), sigma0=5e-3,
# uniform surfactant 0.5, Gibbs elasticity 0.1, Ma=10, Re=1; M_phi=0.1,
# Pi=8.33, Ex=0.16, M_psi=0.01 as in Sec. 6.
CHANNEL_64x128 = dict(
    nx=64, ny=128, walls=1, R=12.0, xb=32.0, yb=40.0, W=4.0, M_phi=0.1,
    rho_A=1.0, rho_ratio=10.0, mu_ratio=1.0, alpha_ratio=1.0, Re=1.0, Ma=10.0,
    sigma0=5e-3, sigma_T=0.0, sigma_TT=1e-3, T_ref=0.5, T_H=1.0, T_C=0.0,
    beta=0.1, Pi=8.33, Ex=0.16, M_psi=0.01, psi0=0.5, Fext_x=0.0, Fext_y=0.0,
    gravity=0.0, nu_A=0.0, alpha_A=0.0, psi_L=0.0, psi_R=0.0, psi_bc=0,
)

# Gibbs elasticity x quadratic sensitivity sweep of the 256x1024 channel.
SWEEP_BETA = (0.05, 0.1, 0.2)
SWEEP_SIGMA_TT = (5e-4, 1e-3, 2e-3)


def channel_64x128() -> dict:
    return copy.deepcopy(CHANNEL_64x128)


def channel_256x1024(beta: float = 0.1, sigma_TT: float = 1e-3) -> dict:
    """256x1024 channel, R=32 a quarter of the way along the wall-bounded axis."""
    p = channel_64x128()
    p.update(nx=256, ny=1024, R=32.0, xb=128.0, yb=256.0, beta=beta, sigma_TT=sigma_TT)
    return p


def channel_256x1024_sweep() -> list[dict]:
    return [channel_256x1024(b, s) for b in SWEEP_BETA for s in SWEEP_SIGMA_TT]


def channel_1024x4096() -> dict:
    """1024x4096 channel, R=96, physics of the 64x128 case."""
    p = channel_64x128()
    p.update(nx=1024, ny=4096, R=96.0, xb=512.0, yb=1024.0)
    return p


def scaled_channel(nx: int, ny: int) -> dict:
    """Channel of arbitrary size with the bubble placed like the 64x128 case
    (R = nx/16*3, centre (nx/2, ny*40/128)); for ragged-size tests."""
    p = channel_64x128()
    p.update(nx=int(nx), ny=int(ny), R=max(3.0, 3.0 * nx / 16.0),
             xb=nx / 2.0, yb=ny * 40.0 / 128.0)
    return p


def _grid(p: dict):
    y, x = np.mgrid[0:p["ny"], 0:p["nx"]]
    return x.astype(np.float64), y.astype(np.float64)


def linear_wall_temperature(p: dict) -> np.ndarray:
    """T_H on the wall plane y=1/2, T_C on y=ny-3/2, linear in between."""
    _, y = _grid(p)
    if not p["walls"]:
        return np.full((p["ny"], p["nx"]), float(p["T_ref"]))
    return p["T_H"] + (p["T_C"] - p["T_H"]) * (y - 0.5) / (p["ny"] - 2.0)


def initial_psi(p: dict) -> np.ndarray:
    """psi0 everywhere, or, with psi_bc 1 or 2 and walls, psi_L on the wall
    plane y=1/2 and psi_R on y=ny-3/2, linear in between (Sec. 2, Sec. 6)."""
    _, y = _grid(p)
    if not p["walls"] or p.get("psi_bc", 0) == 0:
        return np.full((p["ny"], p["nx"]), float(p["psi0"]))
    return p["psi_L"] + (p["psi_R"] - p["psi_L"]) * (y - 0.5) / (p["ny"] - 2.0)


def bubble_fields(p: dict, seed: int | None = None, psi_noise: float = 0.0,
                  u_noise: float = 0.0, T_noise: float = 0.0,
                  p_noise: float = 0.0) -> np.ndarray:
    """Circular bubble (phi = 1 inside) of radius R at (xb, yb) with the
    hyperbolic-tangent interface profile, u = 0, p = 0, linear wall-to-wall T
    and the initial psi of initial_psi, plus optional seeded uniform noise on
    psi, u, T and p."""
    x, y = _grid(p)
    r = np.hypot(x - p["xb"], y - p["yb"])
    out = np.zeros((6, p["ny"], p["nx"]))
    out[0] = 0.5 + 0.5 * np.tanh(2.0 * (p["R"] - r) / p["W"]) if p["R"] > 0 else 0.0
    out[4] = linear_wall_temperature(p)
    out[5] = initial_psi(p)
    if seed is not None:
        rng = np.random.default_rng(seed)
        shape = (p["ny"], p["nx"])
        out[5] += psi_noise * rng.uniform(-1.0, 1.0, shape)
        out[1] += u_noise * rng.uniform(-1.0, 1.0, shape)
        out[2] += u_noise * rng.uniform(-1.0, 1.0, shape)
        out[4] += T_noise * rng.uniform(-1.0, 1.0, shape)
        out[3] += p_noise * rng.uniform(-1.0, 1.0, shape)
    if p["walls"]:
        out[:, 0, :] = 0.0
        out[:, -1, :] = 0.0
    return out


def slab_fields(p: dict, y1: float, y2: float, psi: float | np.ndarray | None = None,
                T: float | None = None) -> np.ndarray:
    """Planar slab of phase B (phi = 1) between y1 and y2 with
    hyperbolic-tangent interfaces, fluid at rest, uniform T and psi."""
    _, y = _grid(p)
    out = np.zeros((6, p["ny"], p["nx"]))
    W = p["W"]
    out[0] = 0.5 * (np.tanh(2.0 * (y - y1) / W) - np.tanh(2.0 * (y - y2) / W))
    out[4] = p["T_ref"] if T is None else T
    out[5] = p["psi0"] if psi is None else psi
    return out


def uniform_fields(p: dict, phi: float = 0.0, T: float | None = None,
                   psi: float | None = None, ux: float = 0.0, uy: float = 0.0,
                   pressure: float = 0.0) -> np.ndarray:
    out = np.zeros((6, p["ny"], p["nx"]))
    out[0] = phi
    out[1] = ux
    out[2] = uy
    out[3] = pressure
    out[4] = p["T_ref"] if T is None else T
    out[5] = p["psi0"] if psi is None else psi
    if p["walls"]:
        out[:, 0, :] = 0.0
        out[:, -1, :] = 0.0
    return out


def parity_fields(p: dict, seed: int = 0) -> np.ndarray:
    """Bubble fields with seeded noise on every field, so that every term of
    the step (velocity-dependent transforms, forces, stencils) is non-zero."""
    return bubble_fields(p, seed=seed, psi_noise=1e-3, u_noise=1e-3, T_noise=1e-3,
                         p_noise=1e-5)


# ---- ensembles and request streams ------------------------------------------------

def ensemble_channels(n: int = 64, seed: int = 0, nx_range=(128, 512), nx_step: int = 16
                      ) -> list[dict]:
    """n independent channels of uneven size and physics: nx uniform over the
    multiples of nx_step in nx_range, ny = 4 nx, bubble R = nx/8 a quarter of
    the way along the channel; Gibbs elasticity beta ~ U(0, 0.3), quadratic
    sensitivity sigma_TT log-uniform in [2e-4, 4e-3], Marangoni number
    Ma ~ U(5, 50); the rest as the 64x128 channel."""
    rng = np.random.default_rng(seed)
    sizes = np.arange(nx_range[0], nx_range[1] + 1, nx_step)
    out = []
    for _ in range(n):
        nx = int(rng.choice(sizes))
        p = channel_64x128()
        p.update(nx=nx, ny=4 * nx, R=nx / 8.0, xb=nx / 2.0, yb=float(nx),
                 beta=float(rng.uniform(0.0, 0.3)),
                 sigma_TT=float(np.exp(rng.uniform(np.log(2e-4), np.log(4e-3)))),
                 Ma=float(rng.uniform(5.0, 50.0)))
        out.append(p)
    return out


def request_stream(n: int = 500, rate: float = 20.0, seed: int = 0, nx_range=(64, 512),
                   fp16_share: float = 0.5, start: str = "quarter") -> list[tuple[float, dict]]:
    """Poisson request arrivals (exponential gaps of mean 1/rate seconds) of
    channels with nx log-uniform in nx_range rounded to a multiple of 16,
    ny = 4 nx, the physics distributions of ensemble_channels, and 16-bit
    population storage with probability fp16_share.  start = "quarter": the
    bubble a quarter of the way along the channel; "reference_plane": a clean
    bubble (beta = 0) on the reference-temperature plane y = ny/2, the
    equilibrium of the self-rewetting law (Sec. 6).  Returns (arrival time in
    seconds, parameters) pairs in arrival order."""
    if start not in ("quarter", "reference_plane"):
        raise ValueError(start)
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += float(rng.exponential(1.0 / rate))
        nx = int(round(np.exp(rng.uniform(np.log(nx_range[0]), np.log(nx_range[1]))) / 16.0)) * 16
        nx = max(nx, 16)
        p = channel_64x128()
        p.update(nx=nx, ny=4 * nx, R=nx / 8.0, xb=nx / 2.0, yb=float(nx),
                 beta=float(rng.uniform(0.0, 0.3)),
                 sigma_TT=float(np.exp(rng.uniform(np.log(2e-4), np.log(4e-3)))),
                 Ma=float(rng.uniform(5.0, 50.0)),
                 precision=1 if rng.uniform() < fp16_share else 0)
        if start == "reference_plane":
            p.update(yb=2.0 * nx, beta=0.0)
        out.append((t, p))
    return out
