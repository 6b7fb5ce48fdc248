"""Seeded synthetic inputs: random vectors and frequency/temperature grids.

Input generators only (shared by the CUDA path and the oracle). The random
initial TPQ vector of the paper (Sec. II.A) is a normalised vector of
complex Gaussian entries, i.e. uniform on the unit sphere of R^{2 N_F}.
Here it is drawn on the host from numpy's seeded generator and handed to
both sides, so parity runs compare the same state element by element.
"""
from __future__ import annotations

import numpy as np


def random_state(n_sites: int, seed: int) -> np.ndarray:
    """Normalised complex Gaussian vector of length 2**n_sites (complex128)."""
    rng = np.random.default_rng(seed)
    d = 1 << n_sites
    v = rng.standard_normal(d) + 1j * rng.standard_normal(d)
    return v / np.linalg.norm(v)


def random_vectors(n_sites: int, n: int, seed: int) -> np.ndarray:
    """n independent unnormalised complex Gaussian vectors, shape [n, 2**N]."""
    rng = np.random.default_rng(seed)
    d = 1 << n_sites
    return rng.standard_normal((n, d)) + 1j * rng.standard_normal((n, d))


def omega_grid(w_min: float, w_max: float, n: int) -> np.ndarray:
    """Uniform grid with both endpoints included."""
    if n == 1:
        return np.array([0.5 * (w_min + w_max)])
    return w_min + (w_max - w_min) * np.arange(n) / (n - 1)


def log_temperatures(t_min: float, t_max: float, n: int) -> np.ndarray:
    return np.exp(np.linspace(np.log(t_min), np.log(t_max), n))
