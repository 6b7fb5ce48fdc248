"""Pins of oracle/cocg3.py (three-term shifted COCG, optional seed switching):
the dense resolvent from LAPACK eigenpairs, the two-term oracle in C, and
seed switching leaving G unchanged. CPU only."""
import numpy as np
import pytest

from ftk_inputs import named, random_state
from oracle import cocg3, dense, sparse


def _case(seed=51):
    cl = named(8)
    K, J = -1.0, 0.1
    dg = dense.Diag(cl, K, J)
    psi = random_state(8, seed)
    q = cl.momenta[1]
    lam = sparse.apply_op(cl, 2, q, psi)
    return cl, K, J, dg, psi, q, lam


def _dense(dg, a, b, z):
    ca, cb = dg.V.T @ a, dg.V.T @ b
    return np.array([np.sum(np.conj(ca) * cb / (zz - dg.E)) for zz in z])


def test_three_term_matches_dense_and_two_term():
    cl, K, J, dg, psi, q, lam = _case()
    z = np.linspace(-3, 3, 61) + 0.05j
    G, it, sw, st = cocg3.shifted_cocg3(cl, K, J, lam, z[30], z, 1e-12, 5000)
    assert st == 0 and sw == 0
    ref = _dense(dg, lam, lam, z)
    assert np.max(np.abs(G - ref)) <= 1e-9 * np.abs(ref).max()
    G2, it2, _, st2 = sparse.cocg(cl, K, J, lam, z[30], z, 1e-12, 5000)
    assert st2 == 0 and np.max(np.abs(G - G2)) <= 1e-9 * np.abs(G2).max()


@pytest.mark.parametrize("seed_z,min_switches,plain_status", [(12 + 8j, 1, 2), (6 + 1j, 2, 0)])
def test_seed_switching_leaves_g_unchanged(seed_z, min_switches, plain_status):
    """A seed far outside the spectrum converges within ~10 iterations; with
    switching the solve moves its seed to the slowest shifts (most of the
    iterations then run on switched seeds) and G stays the resolvent. Without
    switching the farthest seed's r^T r underflows (status 2, the breakdown
    switching avoids); the nearer one still converges and agrees."""
    cl, K, J, dg, psi, q, lam = _case(53)
    z = np.linspace(-4, 12, 81) + 0.05j
    with np.errstate(all="ignore"):
        G0, it0, sw0, st0 = cocg3.shifted_cocg3(cl, K, J, lam, seed_z, z, 1e-11, 20000)
    G1, it1, sw1, st1 = cocg3.shifted_cocg3(cl, K, J, lam, seed_z, z, 1e-11, 20000, switch=True)
    assert st0 == plain_status and sw0 == 0
    assert st1 == 0 and sw1 >= min_switches
    # the switch is exact: the same Krylov iteration continues on the new
    # seed, so it takes as many steps (a wrong scalar transform still
    # converges, on a worse polynomial, in several times more)
    assert it1 <= int(1.1 * it0) + 2
    ref = _dense(dg, lam, lam, z)
    assert np.max(np.abs(G1 - ref)) <= 1e-8 * np.abs(ref).max()
    if plain_status == 0:
        assert np.max(np.abs(G0 - ref)) <= 1e-8 * np.abs(ref).max()


def test_three_term_two_operator_response():
    cl, K, J, dg, psi, q, lam = _case(57)
    a = sparse.apply_op(cl, 0, q, psi)
    z = np.linspace(-2, 2, 41) + 0.1j
    G, it, sw, st = cocg3.shifted_cocg3(cl, K, J, lam, z[20], z, 1e-12, 5000, switch=True, proj=a)
    assert st == 0
    ref = _dense(dg, a, lam, z)
    assert np.max(np.abs(G - ref)) <= 1e-9 * np.abs(ref).max()
