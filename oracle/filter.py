"""Filter operators, equi-energy shells and the filtered-state Green's
function (Sec. II.C and II.D, Eqs. dfilterP, filtered, GAB_TPS). FP64.

TEST INFRASTRUCTURE (see oracle/__init__.py): only tests/ use it.

    P_{g,r,M} v = (1/M) sum_{j=1..M} r e^{i th_j} (r e^{i th_j} + g - H)^{-1} v,
        th_j = 2 pi (j - 1/2) / M                                 (Eq. dfilterP)
    E_m = E_b + (2m + 1) eps, m = 0 .. L-1                        (energy grid)
    phi^m = P_{E_m, eps, M} phi_beta                              (Eq. filtered)
    P(E_m) = <phi^m|phi^m> / (2 eps <phi_beta|phi_beta>)
    G^{AB}(zeta) = sum_m <phi^m| A^dag (zeta + E_m - H)^{-1} B |phi^m>
                   / <phi_beta|phi_beta>                          (Eq. GAB_TPS)
    <O>_b' = sum_m e^{(b - b')E_m} <phi^m|O|phi^m>
             / sum_l e^{(b - b')E_l} <phi^l|phi^l>                (Eq. FRW1)
    P_b'(E_m) = e^{(b - b')E_m} <phi^m|phi^m>
                / (2 eps sum_l e^{(b - b')E_l} <phi^l|phi^l>)     (Eq. FRW2)

Every resolvent is applied by a textbook COCG solve of the complex-symmetric
(z - H) x = b (H real symmetric), one shift at a time, with the oracle's
matrix-free H v; A = B = S^gamma_q (Sec. V).
"""
from __future__ import annotations

import numpy as np

from . import sparse


def contour(gamma: float, rho: float, M: int):
    """Quadrature points z_j = gamma + rho e^{i th_j} and weights
    rho e^{i th_j} / M of Eq. dfilterP."""
    th = 2.0 * np.pi * (np.arange(1, M + 1) - 0.5) / M
    w = rho * np.exp(1j * th)
    return gamma + w, w / M


def solve(cl, K, J, z: complex, b, tol: float = 1e-13, max_iter: int = 20000):
    """x = (z - H)^{-1} b by COCG (bilinear r^T r), to ||r|| <= tol ||b||."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rho = r @ r
    nb = np.linalg.norm(b)
    for _ in range(max_iter):
        ap = z * p - sparse.hv(cl, K, J, p)
        alpha = rho / (p @ ap)
        x += alpha * p
        r -= alpha * ap
        if np.linalg.norm(r) <= tol * nb:
            return x
        rho_new = r @ r
        p = r + (rho_new / rho) * p
        rho = rho_new
    raise RuntimeError("COCG did not converge")


def apply_filter(cl, K, J, phi, gamma: float, rho: float, M: int, tol: float = 1e-13):
    """P_{gamma,rho,M} phi (Eq. dfilterP)."""
    zs, wt = contour(gamma, rho, M)
    out = np.zeros(len(phi), dtype=np.complex128)
    for z, w in zip(zs, wt):
        out += w * solve(cl, K, J, z, phi, tol)
    return out


def energy_grid(e_b: float, eps: float, L: int):
    return e_b + (2 * np.arange(L) + 1) * eps


def filtered_shells(cl, K, J, phi_beta, e_b, eps, L, M, tol=1e-13):
    """[phi^m for m < L] (Eq. filtered)."""
    return [apply_filter(cl, K, J, phi_beta, e, eps, M, tol) for e in energy_grid(e_b, eps, L)]


def probability(shells, phi_beta, eps):
    """P(E_m) = <phi^m|phi^m> / (2 eps <phi_beta|phi_beta>)."""
    nb = np.vdot(phi_beta, phi_beta).real
    return np.array([np.vdot(s, s).real for s in shells]) / (2.0 * eps * nb)


def green(cl, K, J, shells, phi_beta, e_b, eps, gamma_op, q, zetas, tol=1e-13):
    """G(zeta) of Eq. GAB_TPS for A = B = S^gamma_q, one COCG solve per
    (shell, zeta)."""
    nb = np.vdot(phi_beta, phi_beta).real
    grid = energy_grid(e_b, eps, len(shells))
    G = np.zeros(len(zetas), dtype=np.complex128)
    for s, e in zip(shells, grid):
        lam = sparse.apply_op(cl, gamma_op, q, s)
        for i, zeta in enumerate(zetas):
            G[i] += np.vdot(lam, solve(cl, K, J, zeta + e, lam, tol))
    return G / nb


def reweight(o_m, norm2, energies, beta, beta_p, eps):
    """Eqs. FRW1 and FRW2: shells filtered at inverse temperature beta,
    reweighted to beta_p. o_m: [L, ...] the shell expectation values
    <phi^m|O|phi^m> (for a spectrum, -Im G_m(omega) / pi); norm2: [L]
    <phi^m|phi^m>. Returns (<O>_beta_p [...], P_beta_p(E_m) [L]). Numerator
    and denominator share the factor e^{-c}, c = max_m (beta - beta_p) E_m, so
    no exponential overflows."""
    o_m = np.asarray(o_m, dtype=np.float64)
    n = np.asarray(norm2, dtype=np.float64)
    E = np.asarray(energies, dtype=np.float64)
    x = (beta - beta_p) * E
    f = np.exp(x - x.max())
    den = np.sum(f * n)
    o = np.tensordot(f, o_m, axes=(0, 0)) / den
    return o, f * n / (2.0 * eps * den)
