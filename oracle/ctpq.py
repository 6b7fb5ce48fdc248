"""Canonical TPQ state at inverse temperature beta: the Taylor series of
Eq. B1 applied in M_d steps of beta / M_d (Appendix A). FP64.

TEST INFRASTRUCTURE (see oracle/__init__.py): only tests/ use it.

    e^{N beta l / 2} |psi_beta> = e^{N beta (l - h)/2} |psi_0>,  h = H / N,

evaluated as M_d applications of the truncated series
    v <- sum_{k} (tau^k / k!) (l - h)^k v,   tau = N beta / (2 M_d),
with the state renormalised after every step and the logarithms of the
norms accumulated, so that the function returns the unit state and
log || e^{N beta (l - h)/2} psi_0 ||.

M_d (Appendix A): the k-th term is at most X^k / k! with
X = (N beta / 2 M_d)(l + |eps_0|), whose maximum over k is about
e^X / sqrt(2 pi X). Requiring that maximum to be Lambda fixes X as the limit
of X_{j+1} = ln Lambda + (1/2) ln(2 pi X_j), X_0 = Lambda, and
M_d = (N beta / 2)(l + |eps_0|) / X, rounded up (at least 1).

Readings (the paper states neither value): Lambda = 1e4 by default (the
largest term then costs at most ~1e4 ulps of the sum); |eps_0| is the bound
(1/N) sum_b |lambda_min(h_b)| of the lowest eigenvalue of h, from the bond
spectrum (J+K)/4 (twice), (J-K)/4, -(3J+K)/4, so that l + |eps_0| bounds the
spectral radius of l - h for l >= 0. The series of one step stops once a term
falls below 1e-17 of the partial sum past the largest term.
"""
from __future__ import annotations

import math

import numpy as np

from . import sparse


def eps0_bound(cl, K: float, J: float) -> float:
    """|eps_0| <= (1/N) sum_b |lambda_min(h_b)| (bond spectrum of the
    Kitaev-Heisenberg bond h_b = J S_i.S_j + K S^g_i S^g_j)."""
    lmin = min((J + K) / 4, (J - K) / 4, -(3 * J + K) / 4)
    return len(cl.bonds) * abs(lmin) / cl.n_sites


def split_steps(n_sites: int, beta: float, ell: float, eps0_abs: float, lam: float = 1e4):
    """Appendix A: (M_d, X) with X the fixed point of
    X_{j+1} = ln Lambda + (1/2) ln(2 pi X_j) started at X_0 = Lambda."""
    x = float(lam)
    for _ in range(1000):
        nx = math.log(lam) + 0.5 * math.log(2.0 * math.pi * x)
        if abs(nx - x) <= 1e-15 * abs(nx):
            x = nx
            break
        x = nx
    md = max(1, math.ceil(n_sites * beta / 2.0 * (ell + eps0_abs) / x))
    return md, x


def taylor_step(cl, K, J, v, ell, tau):
    """sum_k (tau^k / k!) (l - h)^k v, truncated as stated in the module."""
    n = cl.n_sites
    term = np.array(v, dtype=np.complex128)
    acc = term.copy()
    k = 0
    peak = 0.0
    while True:
        term = (tau / (k + 1)) * (ell * term - sparse.hv(cl, K, J, term) / n)
        acc += term
        k += 1
        tn = float(np.linalg.norm(term))
        peak = max(peak, tn)
        if tn < peak and tn <= 1e-17 * float(np.linalg.norm(acc)):
            return acc
        if k > 10000:
            raise RuntimeError("Taylor series did not converge")


def ctpq_state(cl, K, J, psi0, ell, beta, lam=1e4, md=None):
    """(unit cTPQ state, log || e^{N beta (l - h)/2} psi_0 ||, M_d). md forces
    the number of steps (default: split_steps)."""
    n = cl.n_sites
    if md is None:
        md, _ = split_steps(n, beta, ell, eps0_bound(cl, K, J), lam)
    v = np.array(psi0, dtype=np.complex128)
    nrm = float(np.linalg.norm(v))
    log_norm = math.log(nrm)
    v = v / nrm
    if beta == 0.0:
        return v, log_norm, md
    tau = n * beta / (2.0 * md)
    for _ in range(md):
        v = taylor_step(cl, K, J, v, ell, tau)
        nrm = float(np.linalg.norm(v))
        log_norm += math.log(nrm)
        v = v / nrm
    return v, log_norm, md
