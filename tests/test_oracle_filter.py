"""Pins of oracle/filter.py (Sec. II.C-D). The discrete filter of Eq. dfilterP
has a closed form: the th_j are the M-th roots of -1 (w^M = -1 for
w = e^{i th_j}), and sum over those roots of w / (w - x) = M / (1 + x^M)
(from sum 1/(x - w) = p'(x)/p(x), p = x^M + 1), so in the eigenbasis the
filter multiplies the component of energy E by 1 / (1 + ((E - gamma)/rho)^M).
The COCG-based oracle is checked against that closed form evaluated with
LAPACK eigenpairs of the dense Kronecker-product H. CPU only."""
import numpy as np
import pytest

from ftk_inputs import named, random_state
from oracle import dense, filter as flt


def closed_form(E, gamma, rho, M):
    return 1.0 / (1.0 + ((E - gamma) / rho) ** M)


@pytest.mark.parametrize("M", [4, 8, 16, 32])
def test_contour_sum_closed_form(M):
    """The quadrature of Eq. dfilterP summed in closed form (scalar resolvents)."""
    gamma, rho = -1.3, 0.4
    zs, wt = flt.contour(gamma, rho, M)
    x = np.concatenate([np.linspace(-3, -1.05, 7), np.linspace(-0.95, 0.95, 9), np.linspace(1.05, 3, 7)])
    E = gamma + rho * x
    got = np.array([np.sum(wt / (zs - e)) for e in E])
    assert np.max(np.abs(got - closed_form(E, gamma, rho, M))) <= 1e-12
    assert np.max(np.abs(got.imag)) <= 1e-13


def _setup():
    cl = named(8)
    K, J = -1.0, 0.1
    dg = dense.Diag(cl, K, J)
    phi = random_state(8, 31)
    return cl, K, J, dg, phi


def test_filter_equals_closed_form_in_eigenbasis():
    cl, K, J, dg, phi = _setup()
    gamma, rho, M = float(dg.E[40]), 0.3, 16
    got = flt.apply_filter(cl, K, J, phi, gamma, rho, M)
    c = dg.V.T @ phi
    ref = dg.V @ (closed_form(dg.E, gamma, rho, M) * c)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_filter_keeps_the_window_and_removes_the_rest():
    """M = 32: components with |E - gamma| < rho/2 kept to 3e-10, components
    with |E - gamma| > 2 rho removed to 3e-10 (|x|^M bounds)."""
    cl, K, J, dg, phi = _setup()
    gamma, rho = float(dg.E[100]), 0.25
    got = dg.V.T @ flt.apply_filter(cl, K, J, phi, gamma, rho, 32)
    c = dg.V.T @ phi
    inner = np.abs(dg.E - gamma) < 0.5 * rho
    outer = np.abs(dg.E - gamma) > 2.0 * rho
    assert inner.any() and outer.any()
    assert np.max(np.abs(got[inner] - c[inner])) <= 3e-10 * np.abs(c).max()
    assert np.max(np.abs(got[outer])) <= 3e-10 * np.abs(c).max()


def test_probability_distribution_closed_form():
    cl, K, J, dg, phi = _setup()
    e_b, eps, L, M = float(dg.E[0]) - 0.05, 0.2, 12, 16
    shells = flt.filtered_shells(cl, K, J, phi, e_b, eps, L, M)
    got = flt.probability(shells, phi, eps)
    c2 = np.abs(dg.V.T @ phi) ** 2
    ref = np.array([np.sum(closed_form(dg.E, e, eps, M) ** 2 * c2) for e in flt.energy_grid(e_b, eps, L)])
    ref /= 2 * eps * np.sum(c2)
    assert np.max(np.abs(got - ref)) <= 1e-10 * ref.max()


def test_green_function_closed_form():
    """Eq. GAB_TPS for A = B = S^z_q against the eigenbasis sum
    sum_m sum_mu |<mu|S|phi^m>|^2 / (zeta + E_m - E_mu) / <phi|phi>."""
    cl, K, J, dg, phi = _setup()
    e_b, eps, L, M = float(dg.E[0]) - 0.05, 0.25, 6, 16
    q = cl.momenta[1]
    shells = flt.filtered_shells(cl, K, J, phi, e_b, eps, L, M)
    zetas = np.array([-1.0, 0.0, 0.7]) + 0.1j
    got = flt.green(cl, K, J, shells, phi, e_b, eps, 2, q, zetas)
    S = dg.V.T @ dense.sq_operator(cl, 2, q) @ dg.V
    c = dg.V.T @ phi
    ref = np.zeros(len(zetas), dtype=np.complex128)
    for e in flt.energy_grid(e_b, eps, L):
        a = S @ (closed_form(dg.E, e, eps, M) * c)
        for i, zeta in enumerate(zetas):
            ref[i] += np.sum(np.abs(a) ** 2 / (zeta + e - dg.E))
    ref /= np.vdot(phi, phi).real
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.abs(ref).max()


def test_reweighting_recovers_the_canonical_energy():
    """Eqs. FRW1/FRW2 on a noise-free state: phi_beta = sum_n e^{-beta E_n / 2}|n>
    (every |c_n| = 1), shells of width 2 eps = 0.02 covering the spectrum,
    filter in closed form (M = 32). The discrete filters do not sum to one:
    g(E) = sum_m f_m(E)^2 dips to 1/2 between centres. Reweighted to beta',
    the energy <H> must equal the canonical average with that coverage,
    sum_n g(E_n) e^{-beta' E_n} E_n / sum_n g(E_n) e^{-beta' E_n}, exactly at
    beta' = beta and up to the shell-centre approximation of e^{(beta - beta') E}
    inside a shell otherwise (|beta - beta'| eps ~ 1e-2 relative at most);
    a wrong sign of the exponent misses by far more. FRW2 sums to one."""
    cl = named(8)
    dg = dense.Diag(cl, -1.0, 0.1)
    E = dg.E
    beta, eps, M = 1.0, 0.01, 32
    e_b = E.min() - 10 * eps
    L = int(np.ceil((E.max() - e_b) / (2 * eps))) + 10
    grid = flt.energy_grid(e_b, eps, L)
    c2 = np.exp(-beta * (E - E.min()))                   # |c_n|^2 of phi_beta (rescaled)
    f2 = np.array([closed_form(E, g, eps, M) ** 2 for g in grid])   # [L, n]
    g = f2.sum(axis=0)
    norm2 = f2 @ c2
    h_m = f2 @ (c2 * E)                                  # <phi^m|H|phi^m>
    for beta_p in (0.5, 1.0, 2.0):
        got, P = flt.reweight(h_m, norm2, grid, beta, beta_p, eps)
        w = g * np.exp(-beta_p * (E - E.min()))
        want = np.sum(w * E) / np.sum(w)
        tol = 1e-13 if beta_p == beta else 2 * abs(beta - beta_p) * eps * np.abs(E).max()
        assert abs(got - want) <= tol
        assert abs(np.sum(P) * 2 * eps - 1.0) <= 1e-12
        if beta_p != beta:
            bad, _ = flt.reweight(h_m, norm2, grid, beta, 2 * beta - beta_p, eps)
            assert abs(bad - want) > 10 * tol
