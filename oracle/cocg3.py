"""Shifted COCG in the three-term (residual-only) form, with optional seed
switching. FP64, plain numpy loops over iterations, oracle H v.

TEST INFRASTRUCTURE (see oracle/__init__.py): only tests/ use it.

Seed system (z_s - H) x = lambda, H real symmetric (Sec. II.B; BiCG with
shadow conj(r) = COCG):
    rho_k = r_k^T r_k,  mu_k = r_k^T H r_k,
    alpha_k = rho_k / (z_s rho_k - mu_k - beta_{k-1} rho_k / alpha_{k-1}),
    c_k = beta_{k-1} alpha_k / alpha_{k-1},  beta_k = rho_{k+1} / rho_k,
    r_{k+1} = (1 + c_k) r_k - c_k r_{k-1} - alpha_k (z_s - H) r_k.
Shifted systems z_sigma - H have collinear residuals r^s_k = r_k / pi^s_k:
    pi^s_{k+1} = (1 + alpha_k (z_sigma - z_s)) pi^s_k + c_k (pi^s_k - pi^s_{k-1}),
    alpha^s_k = alpha_k pi^s_k / pi^s_{k+1},
    beta^s_{k-1} = (pi^s_{k-1} / pi^s_k)^2 beta_{k-1},
    p~^s_k = g_k / pi^s_k + beta^s_{k-1} p~^s_{k-1},  G^s += alpha^s_k p~^s_k,
with g_k = proj^dagger r_k (proj = lambda unless given).

Seed switching (Sec. C: the truncation follows the largest shifted
residual; the switch itself is the method of the paper's reference on seed
switching): when the seed's own residual has converged while other shifts
have not, the unconverged shift with the largest ||r_k|| / |pi^s_k| becomes
the seed. Because only residuals enter the recurrences, the switch is exact:
    r_k <- r_k / pi*_k,  r_{k-1} <- r_{k-1} / pi*_{k-1},
    pi^s_k <- pi^s_k / pi*_k,  pi^s_{k-1} <- pi^s_{k-1} / pi*_{k-1},
    alpha_{k-1} <- alpha*_{k-1},  beta_{k-1} <- beta*_{k-1},  rho_k <- rho_k / pi*_k^2,
    z_s <- z*  (g_k / pi^s_k and every shifted residual are unchanged).
Stop when max over unconverged shifts of ||r_k|| / |pi^s_k| <= tol ||lambda||;
a shift is frozen once its own residual is below that bound.
"""
from __future__ import annotations

import numpy as np

from . import sparse


def shifted_cocg3(cl, K, J, lam, z_seed, z, tol, max_iter, switch=False, proj=None):
    """Returns (G [n_shift], iterations, number of seed switches, status):
    0 converged, 1 max_iter, 2 breakdown (r^T r of the seed vanished or
    overflowed: a seed that converges long before the other shifts does this
    without switching)."""
    lam = np.asarray(lam, dtype=np.complex128)
    proj = lam if proj is None else np.asarray(proj, dtype=np.complex128)
    z = np.asarray(z, dtype=np.complex128)
    ns = z.size
    lnorm = np.linalg.norm(lam)
    zs = complex(z_seed)
    r = lam.copy()
    r_prev = np.zeros_like(r)
    rho = r @ r
    alpha_prev, beta_prev = 1.0 + 0j, 0.0 + 0j
    pi_cur = np.ones(ns, dtype=np.complex128)
    pi_prev = np.ones(ns, dtype=np.complex128)
    alpha_s_prev = np.ones(ns, dtype=np.complex128)
    beta_s_prev = np.zeros(ns, dtype=np.complex128)
    pt = np.zeros(ns, dtype=np.complex128)
    G = np.zeros(ns, dtype=np.complex128)
    frozen = np.zeros(ns, dtype=bool)
    switches = 0
    for k in range(max_iter):
        hr = sparse.hv(cl, K, J, r)
        mu = r @ hr
        if k == 0:
            alpha = rho / (zs * rho - mu)
            c = 0.0 + 0j
        else:
            alpha = rho / (zs * rho - mu - beta_prev * rho / alpha_prev)
            c = beta_prev * alpha / alpha_prev
        g = np.vdot(proj, r)
        # shifts
        act = ~frozen
        pi_next = (1.0 + alpha * (z - zs)) * pi_cur + c * (pi_cur - pi_prev)
        alpha_s = alpha * pi_cur / pi_next
        beta_s = (pi_prev / pi_cur) ** 2 * beta_prev if k > 0 else np.zeros(ns, dtype=np.complex128)
        pt = np.where(act, g / pi_cur + beta_s * pt, pt)
        G = np.where(act, G + alpha_s * pt, G)
        # seed residual
        r_next = (1.0 + c) * r - c * r_prev - alpha * (zs * r - hr)
        rho_next = r_next @ r_next
        if rho_next == 0 or not np.isfinite(rho_next) or not np.isfinite(alpha):
            return G, k + 1, switches, 2
        beta = rho_next / rho
        if not np.isfinite(beta):
            return G, k + 1, switches, 2
        r_prev, r = r, r_next
        rho = rho_next
        alpha_s_prev = np.where(act, alpha_s, alpha_s_prev)
        beta_s_prev = np.where(act, beta_s, beta_s_prev)
        pi_prev = np.where(act, pi_cur, pi_prev)
        pi_cur = np.where(act, pi_next, pi_cur)
        alpha_prev, beta_prev = alpha, beta
        rn = np.linalg.norm(r)
        res = rn / np.abs(pi_cur)
        frozen |= res <= tol * lnorm
        if np.all(frozen):
            return G, k + 1, switches, 0
        if switch and rn <= tol * lnorm:
            # the seed has converged, shifts remain: switch to the slowest one
            sw = int(np.argmax(np.where(frozen, -np.inf, res)))
            p_k, p_km1 = pi_cur[sw], pi_prev[sw]
            # beta of the new seed at k (used by the next step): beta_k of sw
            beta_sw = (p_km1 / p_k) ** 2 * beta_prev   # the shifted beta_k relation at the new step
            r = r / p_k
            r_prev = r_prev / p_km1
            rho = rho / p_k ** 2
            alpha_prev = alpha_s_prev[sw]
            beta_prev = beta_sw
            pi_cur = pi_cur / p_k
            pi_prev = pi_prev / p_km1
            zs = complex(z[sw])
            switches += 1
    return G, max_iter, switches, 1
