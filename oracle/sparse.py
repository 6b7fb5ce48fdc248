"""ctypes wrapper of the oracle's plain C routines (oracle/sparse.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU baseline / reference legs; never by the product package.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        cp = C.c_void_p
        _lib.orc_hv.argtypes = [C.c_int, C.c_int, cp, C.c_double, C.c_double, cp, cp]
        _lib.orc_tpq.argtypes = [C.c_int, C.c_int, cp, C.c_double, C.c_double, cp,
                                 C.c_double, C.c_int, C.c_int, cp, cp, cp, cp]
        _lib.orc_tpq.restype = C.c_int
        _lib.orc_apply_op.argtypes = [C.c_int, cp, C.c_int, cp, cp, cp]
        _lib.orc_cocg.argtypes = [C.c_int, C.c_int, cp, C.c_double, C.c_double, cp, C.c_void_p,
                                  C.c_double, C.c_double, C.c_int, cp, C.c_double, C.c_int, C.c_int,
                                  cp, cp, cp]
        _lib.orc_cocg.restype = C.c_int
        _lib.orc_canonical_dsf.argtypes = [C.c_int64, cp, cp, C.c_int, cp, C.c_double,
                                           C.c_int, cp, cp]
        _lib.orc_philox4x32_10.argtypes = [cp, cp, cp]
        _lib.orc_gaussian_state.argtypes = [C.c_int, C.c_uint64, C.c_uint32, cp]
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _bonds(cl):
    return np.ascontiguousarray(cl.bonds, dtype=np.int32)


def hv(cl, K, J, v):
    """H v for the Kitaev-Heisenberg model on cluster cl (Sec. V.A)."""
    v = np.ascontiguousarray(v, dtype=np.complex128)
    out = np.empty_like(v)
    b = _bonds(cl)
    lib().orc_hv(cl.n_sites, cl.n_bonds, _p(b), K, J, _p(v), _p(out))
    return out


def tpq(cl, K, J, psi0, ell, n_steps, save_every):
    """mTPQ iteration; returns (shells [n_saved, D], u, logQ, h2) for k < n_steps."""
    psi0 = np.ascontiguousarray(psi0, dtype=np.complex128)
    n_saved = (n_steps + save_every - 1) // save_every
    shells = np.empty((n_saved, psi0.size), dtype=np.complex128)
    u = np.empty(n_steps); lq = np.empty(n_steps); h2 = np.empty(n_steps)
    b = _bonds(cl)
    got = lib().orc_tpq(cl.n_sites, cl.n_bonds, _p(b), K, J, _p(psi0), ell, n_steps,
                        save_every, _p(shells), _p(u), _p(lq), _p(h2))
    assert got == n_saved
    return shells, u, lq, h2


def apply_op(cl, gamma, q, psi):
    """lambda = S^gamma_q psi (Sec. V)."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(psi)
    pos = np.ascontiguousarray(cl.pos, dtype=np.float64)
    qq = np.ascontiguousarray(q, dtype=np.float64)
    lib().orc_apply_op(cl.n_sites, _p(pos), int(gamma), _p(qq), _p(psi), _p(out))
    return out


def cocg(cl, K, J, lam, z_seed, z, tol, max_iter, unprojected=False, proj=None):
    """Shifted COCG for (z - H) x = lam; returns (G [n_shift], iters,
    rel_resid, status) with G = proj^dagger x (proj None: lam)."""
    lam = np.ascontiguousarray(lam, dtype=np.complex128)
    if proj is not None:
        proj = np.ascontiguousarray(proj, dtype=np.complex128)
    z = np.ascontiguousarray(z, dtype=np.complex128)
    G = np.empty_like(z)
    it = np.zeros(1, dtype=np.int32); res = np.zeros(1)
    b = _bonds(cl)
    st = lib().orc_cocg(cl.n_sites, cl.n_bonds, _p(b), K, J, _p(lam), None if proj is None else _p(proj),
                        float(np.real(z_seed)), float(np.imag(z_seed)), z.size, _p(z),
                        tol, max_iter, int(unprojected), _p(G), _p(it), _p(res))
    return G, int(it[0]), float(res[0]), int(st)


def canonical_dsf(E, a2, omega, eta, temps):
    """Canonical S(q, w, T) from eigenvalues E and a2[n, m] = |<m|S_q|n>|^2 (Eq. chiAB)."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    a2 = np.ascontiguousarray(a2, dtype=np.float64)
    w = np.ascontiguousarray(omega, dtype=np.float64)
    t = np.ascontiguousarray(temps, dtype=np.float64)
    S = np.empty((t.size, w.size))
    lib().orc_canonical_dsf(E.size, _p(E), _p(a2), w.size, _p(w), eta, t.size, _p(t), _p(S))
    return S


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.empty(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def gaussian_state(n_sites, seed, sample=0):
    out = np.empty(1 << n_sites, dtype=np.complex128)
    lib().orc_gaussian_state(n_sites, seed, sample, _p(out))
    return out
