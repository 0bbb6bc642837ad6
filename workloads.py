"""Seeded synthetic workloads shared by the oracle tests, the GPU tests and bench.py.

This module draws random numbers and states grid sizes; it holds none of the
likelihood's arithmetic (no waveform, response, spline, PSD, noise colouring or
cosmology).  Both the oracle side and the CUDA side consume what it returns.

Workloads (shapes and distributions of the paper's injections, Sec. IV, Tables I
and II; the stand-in for the paper's data sets, which are synthetic injections):
  * ``c1``: 1 walker, (2,2) only, K = 256, f in [1e-4, 1e-2] Hz at df = 1/(30 d).
  * ``c2``: 1024 walkers, 6 modes, K = 1024, 1-yr grid f in [1e-5, 1e-1] Hz,
    df = 1/(3.15576e7 s); M_T log-uniform in [1e5, 1e7], q ~ U[0.05, 1],
    a1, a2 ~ U[-0.99, 0.99], z ~ U[1, 8], isotropic sky and orientation,
    t_ref ~ U[0, 3600] s.
  * ``c3``: 8192 walkers, as ``c2`` but M_T log-uniform in [1e3, 1e9].
  * ``c4``: the ``c2`` grid and walkers, injection rescaled in distance.
Walker draws return redshift z in the distance column (column 4); each side
converts z to D_L with its own cosmology.
"""
from __future__ import annotations

import math

import numpy as np

MODES6 = ((2, 2), (3, 3), (4, 4), (2, 1), (3, 2), (4, 3))
YEAR_S = 3.15576e7
DAY_S = 86400.0

# Table I of the paper: uniform prior box of the sampling coordinates
# (ln M_T, q, a1, a2, ln D_L [Gpc], phi_ref, cos iota, lambda, sin beta, psi, ln t_ref [s]).
TABLE1_LOWER = np.array([math.log(1e3), 0.05, -0.99, -0.99, math.log(0.044), 0.0, -1.0, 0.0,
                         -1.0, 0.0, math.log(1.0)])
TABLE1_UPPER = np.array([math.log(1e9), 1.0, 0.99, 0.99, math.log(1298.0), 2 * math.pi, 1.0,
                         2 * math.pi, 1.0, math.pi, math.log(3.15576e8)])

# Parallel-tempered sampler workload: 8 temperatures x 256 walkers around an injection
# with M_T = 2e6 Msun, q = 0.5, z = 3 (angles as Table II's Binary 1; t_ref = 3600 s so
# that the LISA-frame reference time, which differs by up to 500 s, stays positive).
SAMPLER_T, SAMPLER_W = 8, 256
THETA_SAMPLER_Z = (2e6, 0.5, 0.0, 0.0, 3.0, 2.14, 1.05, -0.024 % (2 * math.pi), 0.62, 2.03,
                   3600.0)

# Table II of the paper: Binary, M_T [Msun], q, a1, a2, D_L [Gpc], phi_ref, iota,
# lambda, beta, psi, t_ref [s], SNR (the injections studied in Sec. IV).
TABLE2 = {
    1: (2e6, 1 / 3, 0.0, 0.0, 36.59, 2.14, 1.05, -0.024, 0.62, 2.03, 50.25, 588.0),
    4: (2e6, 1 / 3, 0.85, 0.88, 36.59, 2.14, 1.05, -0.024, 0.62, 2.03, 50.25, 878.0),
    5: (2e6, 1 / 3, -0.83, -0.89, 36.59, 2.14, 1.05, -0.024, 0.62, 2.03, 50.25, 473.0),
    6: (4e7, 1 / 5, 0.0, 0.0, 15.93, 3.10, 1.34, 4.21, -0.73, 0.14, 23.93, 310.0),
    7: (3e5, 7 / 10, 0.0, 0.0, 70.58, 1.22, 1.32, 2.24, -0.22, 2.73, 94.33, 40.0),
}


class Grid:
    """Uniform frequency grid f_j = f0 + j df, j = 0 .. n_bins-1."""

    def __init__(self, f0: float, df: float, n_bins: int):
        self.f0, self.df, self.n_bins = float(f0), float(df), int(n_bins)

    @staticmethod
    def spanning(fmin: float, fmax: float, df: float) -> "Grid":
        return Grid(fmin, df, int(math.floor((fmax - fmin) / df)) + 1)

    def freqs(self) -> np.ndarray:
        return self.f0 + self.df * np.arange(self.n_bins, dtype=np.float64)


GRID_C1 = Grid.spanning(1e-4, 1e-2, 1.0 / (30.0 * DAY_S))
GRID_C2 = Grid.spanning(1e-5, 1e-1, 1.0 / YEAR_S)

# fixed parameters of the single-walker workload (z in the distance column)
THETA_C1_Z = (1e6, 0.2, 0.0, 0.0, 1.0, 1.0, math.pi / 3, 1.0, 0.3, 0.5, 0.0)
T0_C1 = 30.0 * DAY_S   # merger at the end of the 30-day window
T0_YEAR = YEAR_S       # t_coal = t_ref + 1 yr (Sec. II, Table II caption)


def theta_table2(binary: int) -> np.ndarray:
    """The 11 injection parameters of a Table II binary (D_L as printed, in Gpc)."""
    return np.array(TABLE2[binary][:11], dtype=np.float64)


def draw_walkers(B: int, seed: int, logm_range=(5.0, 7.0), tref_max=3600.0) -> np.ndarray:
    """B walkers [B, 11] with redshift z in column 4 (see module docstring)."""
    rng = np.random.default_rng(seed)
    th = np.empty((B, 11), dtype=np.float64)
    th[:, 0] = 10.0 ** rng.uniform(logm_range[0], logm_range[1], B)
    th[:, 1] = rng.uniform(0.05, 1.0, B)
    th[:, 2] = rng.uniform(-0.99, 0.99, B)
    th[:, 3] = rng.uniform(-0.99, 0.99, B)
    th[:, 4] = rng.uniform(1.0, 8.0, B)
    th[:, 5] = rng.uniform(0.0, 2 * math.pi, B)
    th[:, 6] = np.arccos(rng.uniform(-1.0, 1.0, B))
    th[:, 7] = rng.uniform(0.0, 2 * math.pi, B)
    th[:, 8] = np.arcsin(rng.uniform(-1.0, 1.0, B))
    th[:, 9] = rng.uniform(0.0, math.pi, B)
    th[:, 10] = rng.uniform(0.0, tref_max, B)
    return th


def draw_walkers_c2(B: int = 1024, seed: int = 1) -> np.ndarray:
    return draw_walkers(B, seed, (5.0, 7.0))


def draw_walkers_c3(B: int = 8192, seed: int = 3) -> np.ndarray:
    return draw_walkers(B, seed, (3.0, 9.0))


def white_noise(n_bins: int, seed: int = 2) -> np.ndarray:
    """Independent standard normal pairs z[3, n_bins, 2] (channels A, E, T)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((3, n_bins, 2))


def near_injection(theta: np.ndarray, B: int, seed: int, scale: float = 1e-4) -> np.ndarray:
    """B walkers scattered around ``theta`` by relative Gaussian steps (posterior bulk)."""
    rng = np.random.default_rng(seed)
    th = np.repeat(np.asarray(theta, dtype=np.float64)[None, :], B, axis=0)
    th *= 1.0 + scale * rng.standard_normal(th.shape)
    th[:, 1] = np.minimum(th[:, 1], 1.0)
    th[:, 2:4] = np.clip(th[:, 2:4], -0.99, 0.99)
    return th


# Normalizing-flow proposal: 8 affine couplings over the 11 sampling coordinates, each
# with a 2 x 128 hidden-layer network (11 -> 128 -> 128 -> 22).
FLOW_COUPLINGS, FLOW_HIDDEN, FLOW_DIM = 8, 128, 11


def flow_init_weights(seed: int, out_scale: float = 0.0) -> dict:
    """Random starting weights of the flow (uniform +-sqrt(6/fan_in) for the hidden
    layers, zero biases; the output layer scaled by ``out_scale``, 0 = identity flow)."""
    rng = np.random.default_rng(seed)
    C, H, D = FLOW_COUPLINGS, FLOW_HIDDEN, FLOW_DIM
    lim1, lim2, lim3 = math.sqrt(6.0 / D), math.sqrt(6.0 / H), math.sqrt(6.0 / H)
    return {
        "W1": rng.uniform(-lim1, lim1, (C, H, D)).astype(np.float32),
        "b1": np.zeros((C, H), np.float32),
        "W2": rng.uniform(-lim2, lim2, (C, H, H)).astype(np.float32),
        "b2": np.zeros((C, H), np.float32),
        "W3": (out_scale * rng.uniform(-lim3, lim3, (C, 2 * D, H))).astype(np.float32),
        "b3": (out_scale * rng.uniform(-0.1, 0.1, (C, 2 * D))).astype(np.float32),
    }
