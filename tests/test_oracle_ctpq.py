"""Pins of oracle/ctpq.py (cTPQ state by the split Taylor series of Eq. B1,
Appendix A): the exact imaginary-time evolution from a library matrix
exponential of the dense Kronecker H, the fixed point of the step-size
recurrence, independence of the number of steps, beta = 0, and the thermal
energy of reading R1. CPU only."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

from ftk_inputs import named, random_state
from oracle import ctpq, dense, reweight


def test_split_steps_fixed_point():
    """X solves X - (1/2) ln(2 pi X) = ln Lambda; M_d is the smallest integer
    with (N beta/2)(l + |eps_0|)/M_d <= X."""
    for lam in (1e2, 1e4, 1e8):
        for beta in (0.1, 1.0, 10.0, 100.0):
            md, x = ctpq.split_steps(24, beta, 0.5, 0.4, lam)
            assert abs(x - 0.5 * math.log(2 * math.pi * x) - math.log(lam)) <= 1e-12 * x
            need = 24 * beta / 2 * 0.9
            assert md >= 1 and need / md <= x * (1 + 1e-12)
            assert md == 1 or need / (md - 1) > x


def test_eps0_bound_bounds_the_ground_state():
    cl = named(8)
    for K, J in [(-1.0, 0.1), (-1.0, -0.3), (0.0, 1.0)]:
        dg = dense.Diag(cl, K, J)
        assert abs(dg.E[0]) / cl.n_sites <= ctpq.eps0_bound(cl, K, J) + 1e-12


@pytest.mark.parametrize("beta", [0.3, 2.0, 20.0])
def test_ctpq_equals_matrix_exponential(beta):
    """psi_beta = e^{-beta H/2} psi_0 / norm and
    log ||e^{N beta (l - h)/2} psi_0|| = N beta l/2 + log ||e^{-beta H/2} psi_0||,
    against scipy's expm of the dense Kronecker-product H."""
    cl = named(8)
    n = cl.n_sites
    K, J, ell = -1.0, 0.1, 0.5
    psi0 = random_state(n, 21)
    H = dense.hamiltonian(cl, K, J)
    ref = expm(-0.5 * beta * H) @ psi0
    ref_log = n * beta * ell / 2 + math.log(np.linalg.norm(ref))
    ref = ref / np.linalg.norm(ref)
    v, log_norm, md = ctpq.ctpq_state(cl, K, J, psi0, ell, beta)
    assert np.linalg.norm(v - ref) <= 1e-12
    assert abs(log_norm - ref_log) <= 1e-12 * max(1.0, abs(ref_log))
    if beta == 20.0:
        assert md > 1        # the splitting is exercised


def test_number_of_steps_does_not_change_the_state():
    cl = named(8)
    psi0 = random_state(8, 5)
    a, la, _ = ctpq.ctpq_state(cl, -1.0, 0.1, psi0, 0.5, 2.0, md=1)
    b, lb, _ = ctpq.ctpq_state(cl, -1.0, 0.1, psi0, 0.5, 2.0, md=5)
    assert np.linalg.norm(a - b) <= 1e-13 and abs(la - lb) <= 1e-13 * abs(la)


def test_beta_zero_is_the_initial_state():
    cl = named(8)
    psi0 = random_state(8, 3)
    v, log_norm, md = ctpq.ctpq_state(cl, -1.0, 0.1, psi0, 0.5, 0.0)
    assert np.linalg.norm(v - psi0 / np.linalg.norm(psi0)) == 0.0
    assert abs(log_norm - math.log(np.linalg.norm(psi0))) <= 1e-15


def test_energy_matches_reading_r1():
    """<psi_beta|H|psi_beta> of the split series equals R1's reweighting of
    the mTPQ iterates for O = H (both are Eq. B1)."""
    cl = named(8)
    n = cl.n_sites
    K, J, ell = -1.0, 0.1, 0.5
    dg = dense.Diag(cl, K, J)
    psi0 = random_state(n, 11)
    cs, u, lq, h2 = dense.mtpq_eigen(dg, psi0, ell, 400)
    H = dense.hamiltonian(cl, K, J)
    for beta in (0.5, 2.0, 5.0):
        v, _, _ = ctpq.ctpq_state(cl, K, J, psi0, ell, beta)
        e = float(np.real(np.vdot(v, H @ v)))
        o_odd = n * (ell * u - h2 / n ** 2) / (ell - u)
        r1 = reweight.observable(n, ell, u, lq, n * u, o_odd, beta)
        assert abs(e - r1) <= 1e-11 * max(1.0, abs(r1))
