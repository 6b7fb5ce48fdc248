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


# splitmix64 (Steele, Lea and Flood 2014) constants, as unsigned 64-bit values
_GOLDEN = 0x9E3779B97F4A7C15
_MIX1 = 0xBF58476D1CE4E5B9
_MIX2 = 0x94D049BB133111EB


def _as_i64(c: int) -> int:
    return c - (1 << 64) if c >= 1 << 63 else c


def hashed_amplitudes(idx, seed: int, xp=np):
    """Amplitudes at the basis indices idx of an unnormalised vector whose
    every element is a function of (seed, index) alone: re and im uniform in
    [-1/2, 1/2) from the splitmix64 finaliser of seed * 2^40 + 2 idx (+1 for
    im). For vectors too large to draw on the host: the device builds the
    whole vector in slices and a checker evaluates only the elements it
    needs. xp = np (idx int64/uint64, arithmetic in uint64) or torch (idx an
    int64 tensor on any device: the same bits, with wrapping int64 products
    and masked right shifts standing in for the unsigned ones). Returns
    complex128 (numpy) or float64 (re, im) pairs stacked in the last axis
    (torch)."""
    if xp is np:
        x = np.asarray(idx).astype(np.uint64)
        base = np.uint64((seed << 40) & ((1 << 64) - 1))

        def fin(z):
            z = z + np.uint64(_GOLDEN)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(_MIX1)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(_MIX2)
            return z ^ (z >> np.uint64(31))

        with np.errstate(over="ignore"):
            hr = fin(x * np.uint64(2) + base)
            hi = fin(x * np.uint64(2) + base + np.uint64(1))
        scale = 2.0 ** -53
        re = (hr >> np.uint64(11)).astype(np.float64) * scale - 0.5
        im = (hi >> np.uint64(11)).astype(np.float64) * scale - 0.5
        return re + 1j * im
    torch = xp
    x = idx.to(torch.int64)
    base = _as_i64((seed << 40) & ((1 << 64) - 1))

    def srl(z, k):   # logical right shift of the 64-bit pattern
        return (z >> k) & ((1 << (64 - k)) - 1)

    def fin(z):
        z = z + _as_i64(_GOLDEN)
        z = (z ^ srl(z, 30)) * _as_i64(_MIX1)
        z = (z ^ srl(z, 27)) * _as_i64(_MIX2)
        return z ^ srl(z, 31)

    hr = fin(x * 2 + base)
    hi = fin(x * 2 + base + 1)
    scale = 2.0 ** -53
    re = srl(hr, 11).to(torch.float64) * scale - 0.5
    im = srl(hi, 11).to(torch.float64) * scale - 0.5
    return torch.stack([re, im], dim=-1)


def omega_grid(w_min: float, w_max: float, n: int) -> np.ndarray:
    """Uniform grid with both endpoints included."""
    if n == 1:
        return np.array([0.5 * (w_min + w_max)])
    return w_min + (w_max - w_min) * np.arange(n) / (n - 1)


def log_temperatures(t_min: float, t_max: float, n: int) -> np.ndarray:
    return np.exp(np.linspace(np.log(t_min), np.log(t_max), n))
