"""Pins of the oracle's mTPQ iteration (Appendix A), shifted COCG
(Sec. II.B) and Philox generator. CPU only."""
import os

import numpy as np
import pytest

from ftk_inputs import named, random_state, omega_grid
from oracle import dense, sparse

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("n,K,J", [(8, -1.0, 0.1), (12, -1.0, 0.1), (10, -1.0, 0.2)])
def test_tpq_matches_eigenbasis(n, K, J):
    """Matrix-free mTPQ (sparse.c) == the same iteration done exactly in the
    eigenbasis of the Kronecker-product H (u_k, log Q_k, <H^2>_k, shells)."""
    if n == 10:
        from ftk_inputs import honeycomb
        cl = honeycomb((1, 5))
    else:
        cl = named(n)
    dg = dense.Diag(cl, K, J)
    psi0 = random_state(cl.n_sites, 21)
    steps, se = 60, 7
    shells, u, lq, h2 = sparse.tpq(cl, K, J, psi0, 0.5, steps, se)
    cs, u2, lq2, h22 = dense.mtpq_eigen(dg, psi0, 0.5, steps)
    assert np.abs(u - u2).max() < 1e-13
    assert np.abs(lq - lq2).max() < 1e-12
    assert np.abs(h2 - h22).max() < 1e-11
    for s, k in enumerate(range(0, steps, se)):
        assert np.abs(shells[s] - dg.V @ cs[k]).max() < 1e-12
    assert np.all(np.diff(u) <= 1e-15)          # u_k non-increasing (l - h >= 0)


def _dense_green(dg, lam, z):
    c = dg.V.T @ lam
    wt = np.abs(c) ** 2
    return (wt[None, :] / (z[:, None] - dg.E[None, :])).sum(axis=1)


@pytest.mark.parametrize("gamma", [0, 1, 2])
def test_cocg_matches_dense_resolvent(gamma):
    """Shifted COCG G(z) == sum_m |<m|lambda>|^2 / (z - E_m) to the tolerance."""
    cl = named(8)
    K, J = -1.0, 0.1
    dg = dense.Diag(cl, K, J)
    psi = random_state(8, 31 + gamma)
    lam = sparse.apply_op(cl, gamma, cl.momenta[1], psi)
    e0 = -1.2
    z = e0 + omega_grid(-2, 2, 64) + 0.02j
    G, it, res, st = sparse.cocg(cl, K, J, lam, z[32], z, 1e-12, 2000)
    assert st == 0 and it < 2000
    ref = _dense_green(dg, lam, z)
    assert np.abs(G - ref).max() < 1e-9 * np.abs(ref).max()
    assert np.all(G.imag <= 1e-12)


def test_cocg_unprojected_equals_projected():
    """Carrying x^sigma explicitly and projecting at the end gives the same G
    as the projected scalar recurrence (independent check of projection)."""
    cl = named(8)
    psi = random_state(8, 41)
    lam = sparse.apply_op(cl, 2, cl.momenta[2], psi)
    z = -0.5 + omega_grid(-1, 1, 12) + 0.05j
    G1, it1, _, _ = sparse.cocg(cl, -1.0, 0.1, lam, z[3], z, 1e-11, 500, unprojected=False)
    G2, it2, _, _ = sparse.cocg(cl, -1.0, 0.1, lam, z[3], z, 1e-11, 500, unprojected=True)
    assert it1 == it2
    assert np.abs(G1 - G2).max() < 1e-12 * np.abs(G1).max()


def test_cocg_single_shift_is_plain_solve():
    """With one shift equal to the seed, G = lambda^dagger (z - H)^{-1} lambda
    from a dense linear solve."""
    cl = named(6)
    dg = dense.Diag(cl, 0.4, -0.3)
    lam = random_state(6, 2)
    z = np.array([0.3 + 0.1j])
    G, it, _, st = sparse.cocg(cl, 0.4, -0.3, lam, z[0], z, 1e-13, 500)
    x = np.linalg.solve(z[0] * np.eye(64) - dg.h, lam)
    assert st == 0
    assert abs(G[0] - np.vdot(lam, x)) < 1e-11


def test_cocg_not_converged_flag():
    cl = named(8)
    lam = sparse.apply_op(cl, 2, cl.momenta[1], random_state(8, 5))
    z = -1 + omega_grid(-2, 2, 16) + 0.01j
    _, it, res, st = sparse.cocg(cl, -1.0, 0.1, lam, z[8], z, 1e-14, 5)
    assert st == 1 and it == 5 and res > 1e-14


def _kat():
    rows = []
    with open(os.path.join(HERE, "golden", "philox_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            vals = [int(t, 16) for t in line.split()]
            rows.append((vals[:4], vals[4:6], vals[6:10]))
    return rows


def test_philox_known_answers():
    for ctr, key, want in _kat():
        assert sparse.philox4x32_10(ctr, key).tolist() == want


def test_gaussian_state_element_from_the_known_answer():
    """Element 0 of seed 0, sample 0 draws Philox4x32-10 at counter (0, 0, 0, 0)
    and key (0, 0): the first published known-answer vector. Its words give
    u1 = ((w0 << 32 | w1) >> 11 + 1/2) 2^-53 and u2 from (w2, w3), and the
    element is sqrt(-2 ln u1) exp(2 pi i u2) before normalisation: its phase
    is 2 pi u2 whatever the norm. Swapped halves (u1 for u2), a swapped word
    order or a sign slip in the angle all change it."""
    ctr, key, want = _kat()[0]
    assert ctr == [0, 0, 0, 0] and key == [0, 0]
    u1 = ((((want[0] << 32) | want[1]) >> 11) + 0.5) * 2.0 ** -53
    u2 = ((((want[2] << 32) | want[3]) >> 11) + 0.5) * 2.0 ** -53
    for n in (4, 10):
        v = sparse.gaussian_state(n, 0, 0)
        ph = np.angle(v[0]) % (2 * np.pi)
        assert abs(ph - 2 * np.pi * u2) <= 1e-12
    # the angle of the other half (u1) would differ by far more than the bar
    assert 0.0 < u1 < 1.0 and abs(2 * np.pi * u1 - 2 * np.pi * u2) > 0.1


def test_gaussian_state_properties():
    """Normalised; real and imaginary parts i.i.d. with equal variance;
    seed and sample select independent streams."""
    v = sparse.gaussian_state(16, 1234, 0)
    assert abs(np.linalg.norm(v) - 1) < 1e-13
    d = v.size
    re, im = v.real * np.sqrt(2 * d), v.imag * np.sqrt(2 * d)
    assert abs(re.mean()) < 0.02 and abs(im.mean()) < 0.02
    assert abs(re.var() - 1) < 0.03 and abs(im.var() - 1) < 0.03
    assert abs(np.mean(re * im)) < 0.02
    w = sparse.gaussian_state(16, 1234, 1)
    assert abs(np.vdot(v, w)) < 0.02


@pytest.mark.parametrize("unprojected", [False, True])
def test_cocg_two_operator_response(unprojected):
    """A != B: G(z) = <A psi|(z - H)^{-1}|B psi> with A = S^x_q, B = S^z_q
    against the dense resolvent sum_m <A psi|m><m|B psi> / (z - E_m)."""
    cl = named(8)
    K, J = -1.0, 0.1
    dg = dense.Diag(cl, K, J)
    psi = random_state(8, 41)
    q = cl.momenta[1]
    a = sparse.apply_op(cl, 0, q, psi)
    b = sparse.apply_op(cl, 2, q, psi)
    z = np.linspace(-2, 2, 40) + 0.1j
    G, it, res, st = sparse.cocg(cl, K, J, b, z[20], z, 1e-12, 5000, unprojected=unprojected, proj=a)
    assert st == 0
    ca, cb = dg.V.T @ a, dg.V.T @ b
    ref = np.array([np.sum(np.conj(ca) * cb / (zz - dg.E)) for zz in z])
    assert np.max(np.abs(G - ref)) <= 1e-9 * np.abs(ref).max()


def test_cocg_two_operator_reciprocity():
    """(z - H)^{-1} is complex symmetric and R(z)^dagger = R(conj z), so
    G^{AB}(z) = conj(G^{BA}(conj z)), computed by two independent solves."""
    cl = named(8)
    K, J = -1.0, 0.1
    psi = random_state(8, 43)
    q = cl.momenta[2]
    a = sparse.apply_op(cl, 1, q, psi)
    b = sparse.apply_op(cl, 2, q, psi)
    z = np.linspace(-2, 2, 30) + 0.2j
    gab, _, _, s1 = sparse.cocg(cl, K, J, b, z[15], z, 1e-12, 5000, proj=a)
    gba, _, _, s2 = sparse.cocg(cl, K, J, a, np.conj(z[15]), np.conj(z), 1e-12, 5000, proj=b)
    assert s1 == 0 and s2 == 0
    assert np.max(np.abs(gab - np.conj(gba))) <= 1e-9 * np.abs(gab).max()
