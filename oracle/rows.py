"""Sampled rows of the Kitaev-Heisenberg product H v (Sec. V.A), for
clusters where no full product fits a test: (H v)_x for chosen basis states
x, each from the single-site spin matrices, one bond at a time.

TEST INFRASTRUCTURE ONLY: imported by tests/; never by the product package.
Shares no code with the CUDA path.

Matrix elements (basis x = sum_l bit_l 2^l, bit 1 = spin up; S^x, S^y, S^z
as in oracle/dense.py). For a bond (i, j) and y = x with bits i and j
flipped, with s = +1 when bits i and j of x are equal and -1 otherwise:
  <x| S^x_i S^x_j |y> = 1/4
  <x| S^y_i S^y_j |y> = -s/4   (i/2 on an up spin, -i/2 on a down spin:
                                 (+-i/2)^2 = -1/4 for equal spins, +1/4 otherwise)
  <x| S^z_i S^z_j |x> = s/4
so a bond of type gamma adds, to row x,
  diagonal:   (J + K [gamma = z]) s/4 * v_x
  off-diagonal: (J (1 - s)/4 + K ([gamma = x] - s [gamma = y])/4) * v_y.
"""
from __future__ import annotations

import numpy as np


def hv_rows(cl, K: float, J: float, v_at, xs) -> np.ndarray:
    """(H v)_x for every x in xs (int64 array). v_at(idx) returns the
    complex128 amplitudes v at the int64 indices idx."""
    xs = np.asarray(xs, dtype=np.int64)
    out = np.zeros(xs.shape, dtype=np.complex128)
    vx = v_at(xs)
    for i, j, g in np.asarray(cl.bonds).tolist():
        bi = (xs >> i) & 1
        bj = (xs >> j) & 1
        s = np.where(bi == bj, 1.0, -1.0)
        diag = (J + (K if g == 2 else 0.0)) * s / 4
        off = J * (1 - s) / 4 + K * ((1.0 if g == 0 else 0.0) - (s if g == 1 else 0.0)) / 4
        y = xs ^ ((1 << i) | (1 << j))
        out += diag * vx + off * v_at(y)
    return out
