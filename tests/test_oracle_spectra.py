"""Pins of the oracle's canonical spectrum (Sec. III, Eq. chiAB), the
S^gamma_q operator (Sec. V) and the R1 reweighting (Appendix A, Eq. B1).
CPU only."""
import numpy as np
import pytest

from ftk_inputs import honeycomb, named, random_state, omega_grid
from ftk_inputs.lattice import D_X, D_Y, D_Z
from oracle import dense, reweight, sparse

LOR = lambda w, eta: (eta / np.pi) / (w * w + eta * eta)   # noqa: E731


@pytest.mark.parametrize("gamma", [0, 1, 2])
def test_apply_op_matches_kronecker(gamma):
    cl = named(8)
    psi = random_state(8, 5)
    for q in cl.momenta:
        ref = dense.sq_operator(cl, gamma, q) @ psi
        assert np.abs(sparse.apply_op(cl, gamma, q, psi) - ref).max() < 1e-15


def test_dimer_canonical_closed_form():
    """N = 2 dimer, H = L S_A.S_B with L = K + 3J. With S^z at q = (pi, 0)
    (exp(i q.d_z) = -1), S_q = (S^z_A - S^z_B)/sqrt2 links singlet and
    triplet-0 with |<.|S_q|.>|^2 = 1/2: peaks at w = -L (from t0) and +L
    (from s). At q = 0 only the elastic peak of t(+1), t(-1) survives."""
    cl = honeycomb((1, 1))
    K, J, eta = -1.0, 0.2, 0.05
    lam = K + 3 * J
    dg = dense.Diag(cl, K, J)
    w = omega_grid(-2, 2, 81)
    temps = [0.1, 0.5, 2.0]
    es, et = -0.75 * lam, 0.25 * lam
    s_pi = dense.canonical_dsf(dg, 2, [np.pi, 0.0], w, eta, temps)
    s_0 = dense.canonical_dsf(dg, 2, [0.0, 0.0], w, eta, temps)
    for it, t in enumerate(temps):
        z = 3 * np.exp(-et / t) + np.exp(-es / t)
        pt, ps = np.exp(-et / t) / z, np.exp(-es / t) / z
        want_pi = 0.5 * pt * LOR(w - (es - et), eta) + 0.5 * ps * LOR(w - (et - es), eta)
        want_0 = 2 * pt * 0.5 * LOR(w, eta)
        assert np.abs(s_pi[it] - want_pi).max() < 1e-13
        assert np.abs(s_0[it] - want_0).max() < 1e-13


@pytest.mark.parametrize("gamma,dvec", [(0, D_X), (1, D_Y), (2, D_Z)])
def test_kitaev_point_two_parameter_form(gamma, dvec):
    """J = 0 (Kitaev point): <S^a_i S^a_j> vanishes beyond i = j and the
    a-bond (conserved fluxes), so S^a(q, w) = a(w) + b(w) cos(q . d_a) over
    all cluster momenta; a generic J breaks it."""
    cl = named(8)
    w = omega_grid(-1.5, 1.5, 31)
    for J, expect_exact in [(0.0, True), (0.3, False)]:
        dg = dense.Diag(cl, -1.0, J)
        rows = np.array([dense.canonical_dsf(dg, gamma, q, w, 0.05, [0.3])[0] for q in cl.momenta])
        design = np.stack([np.ones(len(cl.momenta)), np.cos(cl.momenta @ dvec)], axis=1)
        coef, *_ = np.linalg.lstsq(design, rows, rcond=None)
        resid = np.abs(design @ coef - rows).max() / np.abs(rows).max()
        if expect_exact:
            assert resid < 1e-12
        else:
            assert resid > 1e-4


def test_heisenberg_point_isotropy():
    """K = 0: SU(2) symmetry makes S^x = S^y = S^z at every momentum."""
    cl = named(8)
    dg = dense.Diag(cl, 0.0, 1.0)
    w = omega_grid(-3, 3, 41)
    for q in cl.momenta:
        s = [dense.canonical_dsf(dg, g, q, w, 0.1, [0.4, 2.0]) for g in range(3)]
        assert np.abs(s[0] - s[2]).max() < 1e-12
        assert np.abs(s[1] - s[2]).max() < 1e-12


def test_sum_rule_canonical():
    """int S(q, w) dw = <S_{-q} S_q>_T. On a finite window the Lorentzian
    tails are removed exactly: each pair contributes
    (1/pi)[atan((w_max - dE)/eta) - atan((w_min - dE)/eta)]."""
    cl = named(8)
    dg = dense.Diag(cl, -1.0, 0.1)
    eta, wmin, wmax = 0.1, -4.0, 4.0
    w = np.linspace(wmin, wmax, 16001)
    for q in cl.momenta[:2]:
        a2 = np.abs(dg.op_eigen(2, q)) ** 2
        for t in [0.2, 1.0]:
            s = dense.canonical_dsf(dg, 2, q, w, eta, [t])[0]
            integral = np.sum((s[1:] + s[:-1]) * 0.5 * np.diff(w))
            p = np.exp(-(dg.E - dg.E[0]) / t)
            p /= p.sum()
            de = dg.E[:, None] - dg.E[None, :]               # E_m - E_n, [m, n]
            frac = (np.arctan((wmax - de) / eta) - np.arctan((wmin - de) / eta)) / np.pi
            want = float(np.sum(a2 * frac * p[None, :]))
            full = dense.canonical_static(dg, 2, q, [t])[0]
            assert abs(integral - want) < 2e-6 * full
            assert abs(want - full) < 0.05 * full      # the window holds most weight


def test_r1_exact_for_energy():
    """R1 applied to O = H reproduces <H> of the canonical TPQ state built
    directly as sum_k (N beta/2)^k/k! (l - h)^k psi_0 (Eq. B1), which in the
    eigenbasis is c_n exp(N beta (l - e_n)/2)."""
    cl = named(8)
    n = cl.n_sites
    dg = dense.Diag(cl, -1.0, 0.1)
    psi0 = random_state(n, 11)
    ell = 0.5
    K = 400
    cs, u, lq, h2 = dense.mtpq_eigen(dg, psi0, ell, K)
    c0 = dg.V.T @ psi0
    for beta in [0.5, 2.0, 5.0]:
        wts = np.abs(c0) ** 2 * np.exp(-beta * (dg.E - dg.E[0]))
        direct = float(wts @ dg.E / wts.sum())
        o_even = n * u
        hbar2 = h2 / n ** 2
        o_odd = n * (ell * u - hbar2) / (ell - u)
        got = reweight.observable(n, ell, u, lq, o_even, o_odd, beta)
        assert abs(got - direct) < 1e-12 * max(1.0, abs(direct))


def test_r1_truncation_flag():
    cl = named(8)
    dg = dense.Diag(cl, -1.0, 0.1)
    psi0 = random_state(8, 3)
    cs, u, lq, h2 = dense.mtpq_eigen(dg, psi0, 0.5, 60)
    steps = np.arange(0, 60, 5)
    _, trunc_hi = reweight.shell_weights(8, 0.5, u, lq, steps, 1.0 / 2.0)
    _, trunc_lo = reweight.shell_weights(8, 0.5, u, lq, steps, 1.0 / 0.005)
    assert not trunc_hi and trunc_lo


def test_shell_green_sum_rule_and_sign():
    """Per shell: -Im G / pi integrates to ||lambda||^2 (exact Lorentzian
    tails removed) and Im G <= 0 for Im z > 0."""
    cl = named(8)
    dg = dense.Diag(cl, -1.0, 0.1)
    psi = random_state(8, 4)
    c = dg.V.T @ psi
    eta = 0.1
    w = np.linspace(-8, 8, 32001)
    q = cl.momenta[1]
    g = dense.shell_green(dg, c, 0, q, w + 1j * eta)
    assert np.all(g.imag <= 0)
    lam = dg.op_eigen(0, q) @ c
    wt = np.abs(lam) ** 2
    frac = (np.arctan((w[-1] - dg.E) / eta) - np.arctan((w[0] - dg.E) / eta)) / np.pi
    s = -g.imag / np.pi
    integral = np.sum((s[1:] + s[:-1]) * 0.5 * np.diff(w))
    assert abs(integral - float(wt @ frac)) < 1e-6 * wt.sum()
    assert abs(wt.sum() - np.linalg.norm(sparse.apply_op(cl, 0, q, psi)) ** 2) < 1e-13


@pytest.mark.slow
def test_estimator_vs_canonical_statistically():
    """The mTPQ-shell estimator (O-DENSE-EST, reading R1) averaged over seeds
    against the canonical spectrum (the paper's Sec. V.B comparison protocol).

    Exact in expectation: the frequency-integrated weight (the static
    structure factor <S_-q S_q>_T). Not exact: the spectral shape. An mTPQ
    state is not a microcanonical shell (the paper says so in Sec. I); its
    energy spread sigma_E (about 0.9 at N = 12) smears every peak, because
    each shell is shifted by its mean energy E_k. The L2 shape error is
    measured and bounded here, not assumed zero; the paper's filtered shells
    remove it."""
    cl = named(12)
    n = cl.n_sites
    dg = dense.Diag(cl, -1.0, 0.1)
    w = omega_grid(-3, 3, 121)
    temps = [0.5, 1.0]
    q = cl.momenta[1]
    canon = dense.canonical_dsf(dg, 2, q, w, 0.05, temps)
    runs = []
    for seed in range(8):
        psi0 = random_state(n, 100 + seed)
        r = dense.dense_estimator(dg, psi0, 0.5, 200, 1, 2, q, w, 0.05, temps)
        assert not r["trunc"].any()
        runs.append(r["S"])
    runs = np.array(runs)
    mean = runs.mean(axis=0)
    dw = w[1] - w[0]
    for it in range(len(temps)):
        ints = runs[:, it].sum(axis=1) * dw
        se = ints.std(ddof=1) / np.sqrt(len(ints))
        want = canon[it].sum() * dw
        assert abs(ints.mean() - want) < 3 * se + 0.02 * want
        rel = np.linalg.norm(mean[it] - canon[it]) / np.linalg.norm(canon[it])
        assert rel < 0.5, rel


@pytest.mark.parametrize("gamma", [0, 1, 2])
def test_detailed_balance_of_the_canonical_weights(gamma):
    """Unbroadened canonical weights: the transition n -> m of S_q at
    omega = E_m - E_n and the reverse transition m -> n of S_{-q} at -omega
    satisfy W_{-q}(m -> n) = e^{-omega/T} W_q(n -> m), since
    S^gamma_{-q} = (S^gamma_q)^dagger and p_m / p_n = e^{-(E_m - E_n)/T}."""
    cl = named(8)
    dg = dense.Diag(cl, -1.0, 0.1)
    q = np.asarray(cl.momenta[1], dtype=float)
    a_p = dg.op_eigen(gamma, q)          # <m|S_q|n>
    a_m = dg.op_eigen(gamma, -q)         # <m|S_-q|n>
    for T in (0.3, 1.0):
        p = np.exp(-(dg.E - dg.E[0]) / T)
        p /= p.sum()
        w_fwd = np.abs(a_p) ** 2 * p[None, :]          # [m, n]: n -> m
        w_rev = (np.abs(a_m) ** 2 * p[None, :]).T      # [m, n]: m -> n under S_-q
        omega = dg.E[:, None] - dg.E[None, :]
        assert np.allclose(w_rev, np.exp(-omega / T) * w_fwd, rtol=1e-10, atol=1e-14)


def test_shell_of_step_is_the_nearest_saved_shell():
    """Brute force: the saved shell nearest to step k, ties to the later one
    (reading R1), clipped to the saved range."""
    steps = [0, 20, 40, 60]
    for k in range(0, 90):
        d = [abs(k - s) for s in steps]
        best = min(d)
        want = max(i for i, x in enumerate(d) if x == best)
        assert int(reweight.shell_of_step(k, steps)) == want


def test_reweighted_spectrum_is_a_convex_combination():
    """R1's shell weights are positive and sum to one: identical shell spectra
    are returned unchanged, and any result lies between the shells' minimum
    and maximum at every frequency."""
    cl = named(8)
    n = cl.n_sites
    dg = dense.Diag(cl, -1.0, 0.1)
    psi0 = random_state(n, 13)
    _, u, lq, _ = dense.mtpq_eigen(dg, psi0, 0.5, 61)
    steps = [0, 20, 40, 60]
    rng = np.random.default_rng(3)
    temps = [0.05, 0.3, 1.0, 3.0]
    same = np.tile(rng.random(17), (4, 1))
    S, _ = reweight.spectrum(n, 0.5, u, lq, steps, same, temps)
    assert np.allclose(S, same[0][None, :], rtol=1e-13, atol=0)
    diff = rng.random((4, 17))
    S, _ = reweight.spectrum(n, 0.5, u, lq, steps, diff, temps)
    assert np.all(S >= diff.min(axis=0) - 1e-14) and np.all(S <= diff.max(axis=0) + 1e-14)
    for t in temps:
        w, _ = reweight.shell_weights(n, 0.5, u, lq, steps, 1.0 / t)
        assert np.all(w >= 0) and abs(w.sum() - 1.0) <= 1e-13
