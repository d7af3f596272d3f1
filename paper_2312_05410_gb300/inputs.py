"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module holds no arithmetic of the time step itself: only parameter sets,
a counter-based random generator and the initial film state.  Both the CUDA
path and the FP64 oracle start from the arrays made here, rounded to FP32 once.

Workload shapes follow the paper's dataset description (Materials and Methods,
"Dataset"): uniform 2D meshes (256x256 in the paper), deposition rate v in
[0.3, 1.0], deposition angle 50-90 degrees, initial phase fraction c_A = 50 %.
The paper's free energy and several closures are deferred to an external
reference, so the default coefficients below are this project's reading
(dimensionless: W = 1, kappa = 2, unit mobilities).

Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used in counter mode: value n of
stream (seed, field) is the SplitMix64 finaliser applied to
key(seed, field) + (n + 1) * golden_gamma.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15

# Stream identifiers for the per-field random draws.
STREAM_C_FILM = 1
STREAM_C_VAPOR = 2
STREAM_ENSEMBLE = 3


def _mix64_scalar(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, field: int) -> int:
    """Key of the counter stream (seed, field)."""
    return _mix64_scalar(_mix64_scalar(seed * GOLDEN_GAMMA + 0x632BE59BD9B4E019) + field * GOLDEN_GAMMA)


def uniform01(seed: int, field: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from counters offset .. offset+n-1 of stream (seed, field)."""
    key = np.uint64(stream_key(seed, field))
    ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = key + ctr * np.uint64(GOLDEN_GAMMA)
    bits = _mix64(z) >> np.uint64(11)
    return bits.astype(np.float64) * (1.0 / 9007199254740992.0)


def truncated_normal(u: np.ndarray, bound: float = 2.0) -> np.ndarray:
    """Standard normal truncated to [-bound, bound] by inverse CDF of u in [0, 1)."""
    from scipy.special import ndtr, ndtri

    lo, hi = ndtr(-bound), ndtr(bound)
    return ndtri(lo + u * (hi - lo))


# --------------------------------------------------------------------------
# Parameter sets.  Field names follow the C struct pf_params (include/pf.h).
# --------------------------------------------------------------------------
PARAM_FIELDS = (
    "dx", "dt", "W_c", "W_phi", "kappa_c", "kappa_phi",
    "MA_bulk", "MB_bulk", "MA_surf", "MB_surf", "sigma_surf",
    "M_phi", "L_phi", "D_rho", "v_mag", "v_angle_deg", "rho_top",
    "phi_mode", "deposition", "diag_every",
)


def default_params(**over) -> dict:
    """Dimensionless model coefficients; dt = 0 means 'caller chooses it'."""
    p = dict(
        dx=1.0, dt=0.0,
        W_c=1.0, W_phi=1.0, kappa_c=2.0, kappa_phi=2.0,
        MA_bulk=1.0, MB_bulk=1.0, MA_surf=0.0, MB_surf=0.0, sigma_surf=0.5,
        M_phi=1.0, L_phi=1.0, D_rho=1.0,
        v_mag=0.5, v_angle_deg=90.0, rho_top=1.0,
        phi_mode=0, deposition=1, diag_every=0,
    )
    for k, v in over.items():
        if k not in p:
            raise KeyError(f"unknown parameter {k}")
        p[k] = v
    return p


@dataclass(frozen=True)
class FilmSpec:
    """Initial film: thickness H cells, film composition c_film +- c_noise (uniform),
    vapor composition c_inc + sigma_v * N(0,1) truncated to +-2 sigma_v."""
    nx: int
    ny: int
    H: float
    seed: int
    c_film: float = 0.5
    c_noise: float = 0.01
    c_inc: float = 0.5
    sigma_v: float = 0.01


# The plain-DNS workloads (sizes and physics of the benchmark configurations).
SMALL_64 = dict(spec=FilmSpec(64, 64, 8.0, seed=0, c_inc=0.5), params=dict(v_mag=0.5), steps=2000)
PAPER_512 = dict(spec=FilmSpec(512, 512, 16.0, seed=1, c_inc=0.5), params=dict(v_mag=0.3, diag_every=1000),
                 steps=50000)


def film_state(spec: FilmSpec, params: dict) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(phi, c, rho) as float32 arrays of shape (ny, nx), x fastest.

    phi: flat film of thickness H in the paper's +-1 convention (solid +1, vapor -1),
    with the equilibrium width sqrt(2) * sqrt(kappa_phi / W_phi) of the double well.
    c: film composition with uniform noise; vapor composition drawn from a
    truncated Gaussian (the paper's interface composition draw).
    rho: vapor density rho_top * (1 - phi) / 2.
    """
    nx, ny = spec.nx, spec.ny
    dx = params["dx"]
    xi = math.sqrt(params["kappa_phi"] / params["W_phi"])
    y = (np.arange(ny, dtype=np.float64) + 0.5) * dx
    prof = -np.tanh((y - spec.H * dx) / (math.sqrt(2.0) * xi))
    phi = np.repeat(prof[:, None], nx, axis=1)
    n = nx * ny
    u_film = uniform01(spec.seed, STREAM_C_FILM, n).reshape(ny, nx)
    u_vap = uniform01(spec.seed, STREAM_C_VAPOR, n).reshape(ny, nx)
    c_film = spec.c_film + spec.c_noise * (2.0 * u_film - 1.0)
    c_vap = spec.c_inc + spec.sigma_v * truncated_normal(u_vap)
    c = np.where(phi >= 0.0, c_film, c_vap)
    rho = params["rho_top"] * (1.0 - phi) * 0.5
    return (phi.astype(np.float32), c.astype(np.float32), rho.astype(np.float32))


def random_state(nx: int, ny: int, seed: int, amp: float = 0.3) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Rough random fields around a film-like state, for stencil checks at odd sizes."""
    n = nx * ny
    a = uniform01(seed, 11, n).reshape(ny, nx)
    b = uniform01(seed, 12, n).reshape(ny, nx)
    r = uniform01(seed, 13, n).reshape(ny, nx)
    phi = 2.0 * a - 1.0
    c = 0.5 + amp * (b - 0.5)
    rho = r
    return (phi.astype(np.float32), c.astype(np.float32), rho.astype(np.float32))


# --------------------------------------------------------------------------
# Ensemble of independent deposition runs (uneven grid sizes, per-run params).
# --------------------------------------------------------------------------
ENSEMBLE_SIDES = (128, 192, 256, 384, 512)


def ensemble_members(n_runs: int = 64, seed: int = 3, v_range=(0.1, 0.9), c_range=(0.3, 0.7),
                     sides=ENSEMBLE_SIDES, H: float = 16.0) -> list[dict]:
    """Per-run grid side, deposition rate and incident composition, all seeded."""
    u = uniform01(seed, STREAM_ENSEMBLE, 3 * n_runs).reshape(n_runs, 3)
    out = []
    for k in range(n_runs):
        side = sides[min(int(u[k, 0] * len(sides)), len(sides) - 1)]
        v = v_range[0] + (v_range[1] - v_range[0]) * u[k, 1]
        ci = c_range[0] + (c_range[1] - c_range[0]) * u[k, 2]
        out.append(dict(nx=side, ny=side, v_mag=float(v), c_inc=float(ci),
                        spec=FilmSpec(side, side, H, seed=seed * 1000 + k, c_inc=float(ci))))
    return out


STREAM_HYBRID = 4
UNET_CHANNELS = (32, 64, 128, 256)
UNET_FDIM = 128
UNET_LB = 3               # look-back frames of (phi, c, rho) fed to the network
UNET_IN = 3 * UNET_LB + 1  # the frames oldest first, then a plane holding dt / dt_ref
UNET_OUT = 3               # increments of (phi, c, rho) of the newest frame


def unet_weights(seed: int = 0) -> dict:
    """Seeded He-normal weights of the time-conditioned U-Net, FP32 arrays in PyTorch layouts
    (conv [Cout, Cin, 3, 3], transposed conv [Cin, Cout, 2, 2]) keyed by layer name.  These are
    untrained random weights: the network is exercised, not fitted."""
    g = np.random.default_rng(seed)
    W = {}

    def he(shape, fan_in):
        return (g.standard_normal(shape) * math.sqrt(2.0 / fan_in)).astype(np.float32)

    W["mlp_w0"] = he((UNET_FDIM, 1), 1)
    W["mlp_b0"] = (g.standard_normal(UNET_FDIM) * 0.5).astype(np.float32)
    W["mlp_w1"] = he((UNET_FDIM, UNET_FDIM), UNET_FDIM)
    W["mlp_b1"] = (g.standard_normal(UNET_FDIM) * 0.1).astype(np.float32)
    W["mlp_w2"] = he((UNET_FDIM, UNET_FDIM), UNET_FDIM)
    W["mlp_b2"] = (g.standard_normal(UNET_FDIM) * 0.1).astype(np.float32)
    for p, c in enumerate(UNET_CHANNELS, 1):
        W[f"proj{p}"] = (g.standard_normal((c, UNET_FDIM)) / math.sqrt(UNET_FDIM)).astype(np.float32)
    cin = UNET_IN
    for p, c in enumerate(UNET_CHANNELS, 1):
        W[f"enc{p}"] = he((c, cin, 3, 3), 9 * cin)
        cin = c
    W["dec4"] = he((256, 256, 3, 3), 9 * 256)
    W["dec3"] = he((128, 256, 3, 3), 9 * 256)
    W["dec2"] = he((64, 128, 3, 3), 9 * 128)
    W["dec1"] = he((32, 64, 3, 3), 9 * 64)
    W["up4"] = he((256, 128, 2, 2), 256)
    W["up3"] = he((128, 64, 2, 2), 128)
    W["up2"] = he((64, 32, 2, 2), 64)
    W["out"] = he((UNET_OUT, 32, 3, 3), 9 * 32)
    for name, c in (("enc1", 32), ("enc2", 64), ("enc3", 128), ("enc4", 256), ("dec4", 256), ("dec3", 128),
                    ("dec2", 64), ("dec1", 32), ("out", UNET_OUT)):
        W[name + "_gamma"] = (1.0 + 0.1 * g.standard_normal(c)).astype(np.float32)
        W[name + "_beta"] = (0.1 * g.standard_normal(c)).astype(np.float32)
    return W


def hybrid_members(n_runs: int = 16, side: int = 256, seed: int = 5, v_range=(0.1, 0.9), c_range=(0.3, 0.7),
                   H: float = 16.0) -> list[dict]:
    """Runs of the hybrid DNS / U-Net workload: equal grids, seeded deposition rate and composition."""
    u = uniform01(seed, STREAM_HYBRID, 2 * n_runs).reshape(n_runs, 2)
    out = []
    for k in range(n_runs):
        v = v_range[0] + (v_range[1] - v_range[0]) * u[k, 0]
        ci = c_range[0] + (c_range[1] - c_range[0]) * u[k, 1]
        out.append(dict(nx=side, ny=side, v_mag=float(v), c_inc=float(ci),
                        spec=FilmSpec(side, side, H, seed=seed * 1000 + k, c_inc=float(ci))))
    return out
