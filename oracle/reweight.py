"""Reweighting of mTPQ shells to temperatures (reading R1), FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper builds the canonical TPQ state from the mTPQ vectors through the
Taylor series of Appendix A, Eq. B1:
    e^{N beta (l - h)/2} |psi_0> = sum_k (N beta/2)^k / k! (l - h)^k |psi_0>,
with (l - h)^k |psi_0> = Q_k |psi_k>. For an observable O that commutes
with H, pairing terms k and k' with k + k' = n and the binomial sum
sum_k 1/(k! (n-k)!) = 2^n / n! give
    <phi_beta|O|phi_beta> = sum_n (N beta)^n / n! <psi_0|(l-h)^n O|psi_0>,
so term n = 2k carries weight w_2k = (N beta)^{2k}/(2k)! Q_k^2 with
O_2k = <psi_k|O|psi_k>, and term n = 2k+1 carries
w_{2k+1} = (N beta)^{2k+1}/(2k+1)! Q_k^2 (l - u_k) with
O_{2k+1} = <psi_k|(l-h) O|psi_k> / (l - u_k).
For the spectrum, O_n is the spectrum of the saved shell nearest to
k = floor(n/2) (ties upward), so shell s receives W_s = sum_{n -> s} w_n.
The paper does not reweight mTPQ shells (its shells are contour-filtered);
this is the reading the build adopts for them. Weights are combined in log
space (log-sum-exp). A truncation flag is raised when the geometric tail
beyond the last term, w_{2K+1} r / (1 - r) with r = N beta (l - u_K)/(2K+2),
exceeds 1e-14 of the total (the paper's 1e-14 cut on the energy
distribution, Sec. III.B).
"""
from __future__ import annotations

import numpy as np
from scipy.special import gammaln, logsumexp


def log_weights(n_sites, ell, u, logQ, beta):
    """log w_n for n = 0 .. 2K-1 (K = len(u))."""
    k = np.arange(len(u))
    lnb = np.log(n_sites * beta)
    le = 2 * k * lnb - gammaln(2 * k + 1) + 2 * logQ
    lo = (2 * k + 1) * lnb - gammaln(2 * k + 2) + 2 * logQ + np.log(ell - u)
    out = np.empty(2 * len(u))
    out[0::2] = le
    out[1::2] = lo
    return out


def shell_of_step(k, shell_steps):
    """Nearest saved shell to step k, ties go to the later shell."""
    se = shell_steps[1] - shell_steps[0] if len(shell_steps) > 1 else 1
    s = np.floor(np.asarray(k) / se + 0.5).astype(np.int64)
    return np.clip(s, 0, len(shell_steps) - 1)


def shell_weights(n_sites, ell, u, logQ, shell_steps, beta):
    """Normalised W_s(beta) and the truncation flag."""
    lw = log_weights(n_sites, ell, u, logQ, beta)
    n = np.arange(lw.size)
    s = shell_of_step(n // 2, shell_steps)
    tot = logsumexp(lw)
    lW = np.full(len(shell_steps), -np.inf)
    for i in range(len(shell_steps)):
        m = s == i
        if m.any():
            lW[i] = logsumexp(lw[m])
    kk = len(u) - 1
    r = n_sites * beta * (ell - u[kk]) / (2 * kk + 2)
    trunc = bool(r >= 1.0 or (lw[-1] + np.log(r / (1 - r)) - tot) > np.log(1e-14))
    return np.exp(lW - tot), trunc


def spectrum(n_sites, ell, u, logQ, shell_steps, S_shell, temps):
    """S(w, T) = sum_s W_s(beta) S_s(w) / sum_s W_s(beta). Returns ([n_T, n_w], trunc[n_T])."""
    S_shell = np.asarray(S_shell, dtype=np.float64)
    out, tr = [], []
    for t in np.atleast_1d(temps):
        w, f = shell_weights(n_sites, ell, u, logQ, shell_steps, 1.0 / t)
        out.append(w @ S_shell)
        tr.append(f)
    return np.array(out), np.array(tr)


def observable(n_sites, ell, u, logQ, O_even, O_odd, beta):
    """sum_n w_n O_n / sum_n w_n with per-step O_2k, O_2k+1 (no shell mapping)."""
    lw = log_weights(n_sites, ell, u, logQ, beta)
    o = np.empty(lw.size)
    o[0::2] = O_even
    o[1::2] = O_odd
    w = np.exp(lw - logsumexp(lw))
    return float(w @ o)
