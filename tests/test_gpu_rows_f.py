"""GPU parity of the rows beyond the mTPQ-shell pipeline, through the C-ABI:
the cTPQ state at chosen beta (Appendix A, Eq. B1 with M_d step splitting),
the two-operator response and seed switching of the shifted solve (Sec. II.B,
Appendix C), and filtered shells with their Green's function and
reweighting (Sec. II.C-D, Eqs. dfilterP, filtered, GAB_TPS, FRW1, FRW2).
Each is compared with the oracle (or the dense resolvent) on the same seeded
inputs. GPU only."""
import numpy as np
import pytest

from ftk_inputs import named, random_state, omega_grid
from oracle import ctpq, dense, filter as flt, sparse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ftk():
    import torch
    from paper_1802_02854_gb300 import build
    assert torch.cuda.is_available()
    build.build()
    import paper_1802_02854_gb300 as m
    m.lib()
    return m


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ------------------------------------------------------------- cTPQ (f2)
@pytest.mark.parametrize("n,beta", [(8, 0.5), (12, 2.0), (12, 0.0), (18, 1.0)])
def test_ctpq_vs_oracle(ftk, n, beta):
    """The cTPQ state at beta, its log norm and M_d against oracle/ctpq.py
    (FP64, 1e-12 relative)."""
    cl = named(n)
    K, J, ell = -1.0, 0.1, 0.5
    psi0 = random_state(n, 5 + n)
    ctx = ftk.Context(cl, K, J, "fp64", max_rhs=1, n_saved=2)
    ctx.set_state(psi0, ell)
    ln, md, en = ctx.ctpq([beta], first_shell=0)
    got = ctx.get_vector(1)
    ctx.close()
    ref, lnr, mdr = ctpq.ctpq_state(cl, K, J, psi0, ell, beta)
    if beta > 0:
        assert md[0] == mdr
    assert rel(got, ref) <= 1e-12
    assert abs(ln[0] - lnr) <= 1e-12 * max(1.0, abs(lnr))
    e_ref = float(np.vdot(ref, sparse.hv(cl, K, J, ref)).real)
    assert abs(en[0] - e_ref) <= 1e-12 * max(1.0, abs(e_ref))


def test_ctpq_beta_ladder(ftk):
    """Ascending betas are reached by increments (each with its own M_d);
    every state and log norm matches the oracle's single-step-sequence state
    at that beta (the step count does not change the state, Appendix A)."""
    cl = named(12)
    K, J, ell = -1.0, 0.1, 0.5
    psi0 = random_state(12, 77)
    betas = [0.25, 1.0, 3.0]
    ctx = ftk.Context(cl, K, J, "fp64", max_rhs=1, n_saved=4)
    ctx.set_state(psi0, ell)
    ln, md, en = ctx.ctpq(betas, first_shell=1)
    steps, energies = ctx.shells()
    for i, b in enumerate(betas):
        ref, lnr, _ = ctpq.ctpq_state(cl, K, J, psi0, ell, b)
        assert rel(ctx.get_vector(2 + i), ref) <= 1e-12
        assert abs(ln[i] - lnr) <= 1e-12 * max(1.0, abs(lnr))
        assert abs(energies[1 + i] - en[i]) == 0.0
    # energies decrease with beta (cooling)
    assert en[0] > en[1] > en[2]
    # the TPQ state is the last cTPQ state
    ref, _, _ = ctpq.ctpq_state(cl, K, J, psi0, ell, betas[-1])
    assert rel(ctx.get_vector(0), ref) <= 1e-12
    ctx.close()


def test_ctpq_checks(ftk):
    cl = named(8)
    ctx = ftk.Context(cl, -1.0, 0.1, "fp64", max_rhs=1, n_saved=2)
    ctx.set_state(random_state(8, 1), 0.5)
    for args in ([[1.0, 0.5]], [[-1.0]], [[1.0], 0.5], [[1.0, 2.0, 3.0]]):
        with pytest.raises(ftk.FtkError) as e:
            ctx.ctpq(*args)
        assert e.value.status == ftk.FTK_EINVAL
    ctx.close()


# ----------------------------------------------- two operators, switching (f3)
def _dense_g(dg, a, b, z):
    ca, cb = dg.V.T @ a, dg.V.T @ b
    return np.array([np.sum(np.conj(ca) * cb / (zz - dg.E)) for zz in z])


@pytest.mark.parametrize("prec", ["fp64", "df", "mixed"])
def test_two_operator_response(ftk, prec):
    """G^{AB}(z) = <S^x_q psi|(z - H)^{-1}|S^z_q psi> (A != B) against the
    oracle's two-term COCG with the same projection vector and the dense
    resolvent."""
    cl = named(12)
    K, J = -1.0, 0.1
    psi0 = random_state(12, 41)
    q = cl.momenta[1]
    ctx = ftk.Context(cl, K, J, prec, max_rhs=2, n_saved=1)
    ctx.set_state(psi0, 0.5)
    ctx.tpq_step(1, 1)
    en = ctx.shells()[1][0]
    ctx.apply_op(0, 2, q, 0)   # B
    ctx.apply_op(0, 0, q, 1)   # A
    omega = omega_grid(-2, 2, 41)
    eta = 0.1
    shifts = omega + 1j * eta
    G, it, sw, st = ctx.shifted_cocg_ex([0], shifts, tol=1e-10, max_iter=5000, proj_slots=[1])
    ctx.close()
    lam_b = sparse.apply_op(cl, 2, q, psi0)
    lam_a = sparse.apply_op(cl, 0, q, psi0)
    z = en + shifts
    Gr, itr, _, str_ = sparse.cocg(cl, K, J, lam_b, z[20], z, 1e-10, 5000, proj=lam_a)
    assert str_ == 0
    tol = 1e-8 if prec != "mixed" else 1e-5
    assert np.abs(G[0] - Gr).max() <= tol * np.abs(Gr).max()
    dg = dense.Diag(cl, K, J)
    want = _dense_g(dg, lam_a, lam_b, z)
    assert np.abs(G[0] - want).max() <= tol * np.abs(want).max()


@pytest.mark.parametrize("prec", ["fp64", "df"])
def test_seed_switching(ftk, prec):
    """A seed far from the spectrum (12 + 8i) converges in a few iterations.
    With switching the solve moves its seed to the slowest shift (exact
    rescaling) and G matches the dense resolvent and the oracle's two-term
    solve seeded in the middle of the grid at every shift, in about as many
    iterations as without switching (where the range guard carries the
    converged seed instead)."""
    cl = named(8)
    K, J = -1.0, 0.1
    psi = random_state(8, 53)
    q = cl.momenta[1]
    lam = sparse.apply_op(cl, 2, q, psi)
    z = np.concatenate([np.linspace(-4, 12, 81) + 0.05j, [12 + 8j]])
    ctx = ftk.Context(cl, K, J, prec, max_rhs=1, n_saved=1)
    ctx.set_probe(0, lam, 0.0)
    G0, it0, sw0, _ = ctx.shifted_cocg_ex([0], z, tol=1e-11, max_iter=20000, seed_index=81)
    G1, it1, sw1, _ = ctx.shifted_cocg_ex([0], z, tol=1e-11, max_iter=20000, seed_index=81, seed_switch=True)
    ctx.close()
    assert sw0[0] == 0 and sw1[0] >= 1
    assert it1[0] <= int(1.1 * it0[0]) + 2
    dg = dense.Diag(cl, K, J)
    ref = _dense_g(dg, lam, lam, z)
    for G in (G0, G1):
        assert np.abs(G[0] - ref).max() <= 1e-8 * np.abs(ref).max()
    Gr, itr, _, st = sparse.cocg(cl, K, J, lam, z[40], z[:81], 1e-11, 20000)
    assert st == 0
    assert np.abs(G1[0, :81] - Gr).max() <= 1e-8 * np.abs(Gr).max()


def test_switching_in_a_block(ftk):
    """Switching is per right-hand side: a block of two probes, one of which
    switches, gives the single-probe results."""
    cl = named(8)
    K, J = -1.0, 0.1
    psi = random_state(8, 3)
    q = cl.momenta[2]
    lams = [sparse.apply_op(cl, g, q, psi) for g in (2, 0)]
    z = np.concatenate([np.linspace(-3, 3, 31) + 0.1j, [9 + 6j]])
    ctx = ftk.Context(cl, K, J, "fp64", max_rhs=2, n_saved=1)
    ctx.set_probe(0, lams[0], 0.0)
    ctx.set_probe(1, lams[1], 0.0)
    Gb, itb, swb, _ = ctx.shifted_cocg_ex([0, 1], z, tol=1e-11, max_iter=10000, seed_index=31, seed_switch=True)
    for j in range(2):
        Gs, its, sws, _ = ctx.shifted_cocg_ex([j], z, tol=1e-11, max_iter=10000, seed_index=31, seed_switch=True)
        assert np.abs(Gb[j] - Gs[0]).max() <= 1e-10 * np.abs(Gs[0]).max()
        assert swb[j] == sws[0] >= 1
    ctx.close()


def test_graph_reuse_across_solves(ftk):
    """Solves of different shapes in a row (the cached graph is updated or
    re-instantiated) give the results of fresh contexts."""
    cl = named(10)
    K, J = -1.0, 0.1
    psi = random_state(10, 9)
    lam = sparse.apply_op(cl, 2, cl.momenta[1], psi)
    cases = [(omega_grid(-2, 2, 33), 0.1), (omega_grid(-2, 2, 65), 0.05), (omega_grid(-1, 1, 33), 0.1)]
    ctx = ftk.Context(cl, K, J, "fp64", max_rhs=2, n_saved=1)
    ctx.set_probe(0, lam, 0.0)
    ctx.set_probe(1, lam, 0.0)
    got = [ctx.shifted_cocg([0], om, eta, tol=1e-10)[0] for om, eta in cases]
    got.append(ctx.shifted_cocg([0, 1], cases[0][0], cases[0][1], tol=1e-10)[0][1])
    ctx.close()
    for i, ((om, eta), g) in enumerate(zip(cases + [cases[0]], got)):
        fresh = ftk.Context(cl, K, J, "fp64", max_rhs=1, n_saved=1)
        fresh.set_probe(0, lam, 0.0)
        want = fresh.shifted_cocg([0], om, eta, tol=1e-10)[0]
        fresh.close()
        if i < len(cases):
            # the same plan and inputs: the same arithmetic, bit for bit
            assert np.array_equal(np.ravel(g), np.ravel(want))
        else:
            # a block of two runs another H.V plan (rounding order)
            assert np.abs(np.ravel(g) - np.ravel(want)).max() <= 1e-10 * np.abs(want).max()


# ------------------------------------------------------ filter shells (f1)
def test_filter_pipeline_vs_oracle(ftk):
    """cTPQ state at beta -> L filtered shells (Eq. filtered, M = 16) -> S^z_q
    probes -> Green's function per shell (Eq. GAB_TPS) -> reweighting to other
    temperatures (Eqs. FRW1, FRW2), every stage against the oracle on the
    same seeded state: shells and their norms to 1e-9, G to 1e-8, S and P to
    1e-8."""
    cl = named(8)
    K, J, ell = -1.0, 0.1, 0.5
    psi0 = random_state(8, 11)
    beta = 1.0
    dg = dense.Diag(cl, K, J)
    e_b, eps, L, M = float(dg.E[0]) - 0.05, 0.25, 6, 16
    ctx = ftk.Context(cl, K, J, "fp64", max_rhs=1, n_saved=1 + L)
    ctx.set_state(psi0, ell)
    ctx.ctpq([beta], first_shell=0)
    n2, it = ctx.filter_shells(1, e_b, eps, L, M, tol=1e-12, max_iter=4000, first_shell=1)
    phi, _, _ = ctpq.ctpq_state(cl, K, J, psi0, ell, beta)
    shells = flt.filtered_shells(cl, K, J, phi, e_b, eps, L, M, tol=1e-13)
    for m in range(L):
        assert rel(ctx.get_vector(2 + m), shells[m]) <= 1e-9
    n2_ref = np.array([np.vdot(s, s).real for s in shells])
    assert np.abs(n2 - n2_ref).max() <= 1e-9 * n2_ref.max()
    steps, energies = ctx.shells()
    grid = flt.energy_grid(e_b, eps, L)
    assert np.abs(energies[1:] - grid).max() <= 1e-14
    q = cl.momenta[1]
    omega = omega_grid(-2, 2, 24)
    eta = 0.1
    G = []
    for m in range(L):
        ctx.apply_op(1 + m, 2, q, 0)
        g, _, _ = ctx.shifted_cocg([0], omega, eta, tol=1e-11, max_iter=4000)
        G.append(g[0])
    G = np.array(G)
    G_ref = np.array([flt.green(cl, K, J, [shells[m]], phi, e_b + 2 * m * eps, eps, 2, q, omega + 1j * eta)
                      for m in range(L)])
    assert np.abs(G - G_ref).max() <= 1e-8 * np.abs(G_ref).max()
    T = np.array([0.5, 1.0, 2.0])
    S, P = ctx.filter_spectrum(G, grid, n2, beta, eps, T)
    ctx.close()
    for t, temp in enumerate(T):
        s_ref, p_ref = flt.reweight(-G_ref.imag / np.pi, n2_ref, grid, beta, 1.0 / temp, eps)
        assert rel(S[t], s_ref) <= 1e-8
        assert rel(P[t], p_ref) <= 1e-8


def test_filter_equals_closed_form_on_the_gpu(ftk):
    """The GPU filter of a random state against the closed form of the
    discrete filter in the eigenbasis, 1 / (1 + ((E - E_m)/eps)^M) (LAPACK
    eigenpairs), at N = 10 with 8 shells of M = 32 points."""
    cl = named(10)
    K, J = -1.0, 0.1
    phi = random_state(10, 19)
    dg = dense.Diag(cl, K, J)
    e_b, eps, L, M = float(dg.E[0]) - 0.1, 0.15, 8, 32
    ctx = ftk.Context(cl, K, J, "fp64", max_rhs=1, n_saved=L)
    ctx.set_state(phi, 0.5)
    n2, it = ctx.filter_shells(0, e_b, eps, L, M, tol=1e-12, max_iter=6000, first_shell=0)
    c = dg.V.T @ phi
    for m, em in enumerate(flt.energy_grid(e_b, eps, L)):
        f = 1.0 / (1.0 + ((dg.E - em) / eps) ** M)
        want = dg.V @ (f * c)
        assert rel(ctx.get_vector(1 + m), want) <= 1e-9
        assert abs(n2[m] - np.sum(np.abs(f * c) ** 2)) <= 1e-9 * max(n2[m], 1e-300) + 1e-15
    ctx.close()


def test_filter_checks(ftk):
    cl = named(8)
    ctx = ftk.Context(cl, -1.0, 0.1, "df", max_rhs=1, n_saved=4)
    ctx.set_state(random_state(8, 1), 0.5)
    with pytest.raises(ftk.FtkError) as e:
        ctx.filter_shells(0, -2.0, 0.2, 2, 16)
    assert e.value.status == ftk.FTK_EINVAL   # needs FTK_FP64
    ctx.close()
    ctx = ftk.Context(cl, -1.0, 0.1, "fp64", max_rhs=1, n_saved=4)
    ctx.set_state(random_state(8, 1), 0.5)
    with pytest.raises(ftk.FtkError):
        ctx.filter_shells(0, -2.0, 0.2, 8, 16)   # more shells than n_saved
    with pytest.raises(ftk.FtkError):
        ctx.filter_shells(0, -2.0, 0.2, 2, 33)   # M > 32
    assert ftk.ftk_filter_footprint(128, 16, 100) > 0 and ftk.ftk_filter_footprint(300, 16, 100) == 0
    ctx.close()
