"""Dense oracles (numpy/scipy LAPACK, N <= 12).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU legs; never by the product package. Shares no code with the
CUDA path.

* ``hamiltonian``: the Kitaev-Heisenberg H of Sec. V.A built from Kronecker
  products of spin-1/2 matrices, independent of any bit-manipulation rule.
* ``canonical_dsf``: O-DENSE-CANON, the canonical finite-temperature
  spectrum of Sec. III, Eq. 'chiAB', by full diagonalisation.
* ``dense_estimator``: O-DENSE-EST, the estimator the CUDA path computes
  (mTPQ shells, per-shell Green's functions, reweighting), evaluated exactly
  in the eigenbasis without any Krylov solver.

Basis convention (Sec. II.A): x = sum_l bit_l 2^l, bit 1 = spin up. In a
Kronecker product the first factor is the most significant bit, so site l is
factor N-1-l. Single-site order (down, up):
    S^x = [[0, 1], [1, 0]]/2,  S^y = [[0, i], [-i, 0]]/2,  S^z = diag(-1, 1)/2
(S^y |up> = (i/2)|down>, S^y |down> = (-i/2)|up>).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import reweight as _rw
from . import sparse as _sparse

SX = np.array([[0, 1], [1, 0]], dtype=np.complex128) / 2
SY = np.array([[0, 1j], [-1j, 0]], dtype=np.complex128) / 2
SZ = np.array([[-1, 0], [0, 1]], dtype=np.complex128) / 2
SPIN = (SX, SY, SZ)


def site_op(n_sites: int, l: int, op: np.ndarray) -> sp.csr_matrix:
    """op acting on site l, identity elsewhere (sparse, complex)."""
    out = sp.identity(1, dtype=np.complex128, format="csr")
    for f in range(n_sites - 1, -1, -1):          # most significant factor first
        out = sp.kron(out, sp.csr_matrix(op) if f == l else sp.identity(2, format="csr"),
                      format="csr")
    return out


def hamiltonian_sparse(cl, K: float, J: float) -> sp.csr_matrix:
    """Sparse H = sum_<ij>_gamma J S_i.S_j + K S^gamma_i S^gamma_j (Sec. V.A)."""
    n = cl.n_sites
    ops = [[site_op(n, l, SPIN[a]) for a in range(3)] for l in range(n)]
    h = sp.csr_matrix((1 << n, 1 << n), dtype=np.complex128)
    for i, j, g in cl.bonds:
        for a in range(3):
            h = h + J * (ops[i][a] @ ops[j][a])
        h = h + K * (ops[i][g] @ ops[j][g])
    return h


def hamiltonian(cl, K: float, J: float, real: bool = True) -> np.ndarray:
    """Dense H = sum_<ij>_gamma J S_i.S_j + K S^gamma_i S^gamma_j (Sec. V.A)."""
    h = hamiltonian_sparse(cl, K, J).toarray()
    if real:
        if np.abs(h.imag).max() > 0:
            raise AssertionError("Kitaev-Heisenberg H must be real in the S^z basis")
        return h.real.copy()
    return h


def sq_operator_sparse(cl, gamma: int, q) -> sp.csr_matrix:
    """S^gamma_{+Q} = N^{-1/2} sum_l exp(i Q.R_l) S^gamma_l (Sec. V), sparse."""
    n = cl.n_sites
    q = np.asarray(q, dtype=np.float64)
    acc = sp.csr_matrix((1 << n, 1 << n), dtype=np.complex128)
    for l in range(n):
        acc = acc + np.exp(1j * float(q @ cl.pos[l])) * site_op(n, l, SPIN[gamma])
    return acc / np.sqrt(n)


def sq_operator(cl, gamma: int, q) -> np.ndarray:
    """Dense S^gamma_{+Q}."""
    return sq_operator_sparse(cl, gamma, q).toarray()


class Diag:
    """Eigen-decomposition of the dense H (LAPACK eigh)."""

    def __init__(self, cl, K, J):
        self.cl, self.K, self.J = cl, K, J
        self.h = hamiltonian(cl, K, J)
        self.E, self.V = np.linalg.eigh(self.h)

    def op_eigen(self, gamma, q) -> np.ndarray:
        """<m|S_q|n> in the eigenbasis."""
        a = sq_operator_sparse(self.cl, gamma, q)
        re = self.V.T @ (a.real @ self.V)
        im = self.V.T @ (a.imag @ self.V)
        return re + 1j * im


def canonical_dsf(dg: Diag, gamma, q, omega, eta, temps) -> np.ndarray:
    """O-DENSE-CANON (Sec. III, Eq. 'chiAB' with A = B = S^gamma_q):
    S(w, T) = sum_{n,m} e^{-E_n/T}/Z |<m|S_q|n>|^2 (eta/pi)/((w - E_m + E_n)^2 + eta^2).
    Returns [n_T, n_w]."""
    a = dg.op_eigen(gamma, q)
    a2 = np.abs(a) ** 2            # a2[m, n]
    return _sparse.canonical_dsf(dg.E, np.ascontiguousarray(a2.T), omega, eta, temps)


def canonical_static(dg: Diag, gamma, q, temps) -> np.ndarray:
    """<S_{-Q} S_{+Q}>_T = sum_n p_n sum_m |<m|S_q|n>|^2 (the sum rule's right side)."""
    a2 = np.abs(dg.op_eigen(gamma, q)) ** 2
    out = []
    for t in np.atleast_1d(temps):
        p = np.exp(-(dg.E - dg.E[0]) / t)
        p /= p.sum()
        out.append(float(p @ a2.sum(axis=0)))
    return np.array(out)


def mtpq_eigen(dg: Diag, psi0, ell, n_steps):
    """mTPQ in the eigenbasis (Appendix A building block, exact):
    c^{k+1} = (l - e) c^k / q_k with e = E/N; u_k = sum |c^k_n|^2 e_n,
    logQ_k = sum_{k'<k} log q_k', h2_k = <psi_k|H^2|psi_k>.
    Returns (coefficients [n_steps, D] of psi_k in the eigenbasis, u, logQ, h2)."""
    n = dg.cl.n_sites
    e = dg.E / n
    c = dg.V.T @ np.asarray(psi0, dtype=np.complex128)
    cs, u, lq, h2 = [], [], [], []
    acc = 0.0
    for _ in range(n_steps):
        p = np.abs(c) ** 2
        cs.append(c.copy())
        u.append(float(p @ e))
        lq.append(acc)
        h2.append(float(p @ dg.E ** 2))
        c = (ell - e) * c
        q = np.linalg.norm(c)
        acc += np.log(q)
        c = c / q
    return np.array(cs), np.array(u), np.array(lq), np.array(h2)


def shell_green(dg: Diag, coeff, gamma, q, z, a=None) -> np.ndarray:
    """G(z) = <lambda|(z - H)^{-1}|lambda>, lambda = S_q psi, in the eigenbasis:
    sum_m |<m|lambda>|^2 / (z - E_m) (Sec. II.B, G^{AB} with A = B).
    a: optional precomputed <m|S_q|n>."""
    if a is None:
        a = dg.op_eigen(gamma, q)
    lam = a @ coeff
    w = np.abs(lam) ** 2
    z = np.asarray(z, dtype=np.complex128)
    return (w[None, :] / (z[:, None] - dg.E[None, :])).sum(axis=1)


def dense_estimator(dg: Diag, psi0, ell, n_steps, save_every, gamma, q, omega, eta, temps):
    """O-DENSE-EST: the mTPQ-shell FTKomega estimator evaluated exactly.

    Shells psi_k for k % save_every == 0 (k < n_steps); per shell the Green's
    function at z = E_k + w + i eta with E_k = N u_k; spectra
    S_s(w) = -Im G_s / pi; temperatures by reweighting R1 (oracle.reweight).
    Returns dict with u, logQ, h2, shell_steps, G [n_s, n_w], S [n_T, n_w], trunc [n_T].
    """
    n = dg.cl.n_sites
    cs, u, lq, h2 = mtpq_eigen(dg, psi0, ell, n_steps)
    steps = np.arange(0, n_steps, save_every)
    omega = np.asarray(omega, dtype=np.float64)
    a = dg.op_eigen(gamma, q)
    G = np.array([shell_green(dg, cs[k], gamma, q, n * u[k] + omega + 1j * eta, a) for k in steps])
    S, trunc = _rw.spectrum(n, ell, u, lq, steps, -G.imag / np.pi, temps)
    return dict(u=u, logQ=lq, h2=h2, shell_steps=steps, G=G, S=S, trunc=trunc)
