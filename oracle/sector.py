"""Momentum sectors of the translation group, written from the definitions.
FP64, numpy.

TEST INFRASTRUCTURE (see oracle/__init__.py): only tests/ use it.

A group of site permutations g acts on basis states, g|x> = |g.x> with bit
g(l) of g.x equal to bit l of x. For a one-dimensional character chi of the
group (chi(g) = exp(-i Q.a_g) for the translation by a_g at momentum Q) the
projector is P = (1/|G|) sum_g chi(g)^* g. Every orbit has the representative
r = min_g g.r; P|r> is nonzero exactly when chi = 1 on the stabiliser of r,
and then the sector basis vector is |r> = P|r> / ||P|r>|| with
||P|r>||^2 = 1/o_r (o_r the orbit size), i.e. |r> = sqrt(o_r) P|r>.

The functions build that basis literally (as full-space vectors) and give
  basis(...)    -> representatives and the matrix B [2^N, d] of basis columns
  block(...)    -> the sector block B^dag H B of the dense Kronecker H
  embed/project -> B v and B^dag psi without forming B (any N: one term per
                   (representative, group element))
"""
from __future__ import annotations

import numpy as np


def act(x, perm):
    """g.x for integer states x (numpy array) and the site permutation perm."""
    x = np.asarray(x, dtype=np.int64)
    y = np.zeros_like(x)
    for l, t in enumerate(perm):
        y |= ((x >> l) & 1) << int(t)
    return y


def inverse(perm):
    inv = np.empty_like(np.asarray(perm))
    inv[np.asarray(perm)] = np.arange(len(perm))
    return inv


def representatives(n_sites, perms, chi):
    """(reps ascending, orbit sizes) of the orbits on whose stabiliser chi is 1."""
    x = np.arange(1 << n_sites, dtype=np.int64)
    imgs = np.stack([act(x, p) for p in perms])            # [n_g, 2^N]
    rep = imgs.min(axis=0)
    is_rep = rep == x
    r = x[is_rep]
    fixed = imgs[:, is_rep] == r[None, :]                  # stabiliser membership [n_g, n_rep]
    chi = np.asarray(chi, dtype=np.complex128)
    ok = np.all(np.where(fixed, np.abs(chi[:, None] - 1.0) < 1e-9, True), axis=0)
    orbit = len(perms) // fixed.sum(axis=0)
    return r[ok], orbit[ok]


def basis(n_sites, perms, chi):
    """(reps, B [2^N, d]) with B[:, i] = sqrt(o_r) P|r_i>."""
    reps, orbit = representatives(n_sites, perms, chi)
    chi = np.asarray(chi, dtype=np.complex128)
    B = np.zeros((1 << n_sites, len(reps)), dtype=np.complex128)
    for g, p in enumerate(perms):
        np.add.at(B, (act(reps, p), np.arange(len(reps))), np.conj(chi[g]))
    B *= np.sqrt(orbit)[None, :] / len(perms)
    return reps, B


def block(H, B):
    """The sector block B^dag H B (Hermitian)."""
    return B.conj().T @ (H @ B)


def project(psi, reps, orbit, perms, chi):
    """B^dag psi: <r| psi = (sqrt(o_r)/|G|) sum_h chi(h)^* psi[h^{-1}.r]."""
    chi = np.asarray(chi, dtype=np.complex128)
    out = np.zeros(len(reps), dtype=np.complex128)
    for h, p in enumerate(perms):
        out += np.conj(chi[h]) * psi[act(reps, inverse(p))]
    return out * np.sqrt(orbit) / len(perms)


def embed(v, reps, orbit, perms, chi, n_sites):
    """B v: sum_r v_r sqrt(o_r)/|G| sum_h chi(h)^* |h.r>."""
    chi = np.asarray(chi, dtype=np.complex128)
    out = np.zeros(1 << n_sites, dtype=np.complex128)
    coef = np.asarray(v) * np.sqrt(orbit) / len(perms)
    for h, p in enumerate(perms):
        np.add.at(out, act(reps, p), np.conj(chi[h]) * coef)
    return out
