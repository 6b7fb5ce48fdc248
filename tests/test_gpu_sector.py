"""GPU parity of the momentum-sector path (translation symmetry), through
the C-ABI, against oracle/sector.py (the sector basis from its definition and
the dense or matrix-free full-space H) and the oracle's full-basis estimator:
sector dimension and representatives, projection, sector H.v, the Hermitian
Lanczos Green's function, and the whole mTPQ -> S^z_q -> G -> spectrum
pipeline run sector by sector and merged. GPU only."""
import numpy as np
import pytest

from ftk_inputs import named, random_state, omega_grid, translations, characters
from oracle import dense, sector, sparse

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


@pytest.mark.parametrize("n", [8, 12])
def test_sector_basis_projection_and_hv(ftk, n):
    cl = named(n)
    K, J = -1.0, 0.1
    H = dense.hamiltonian(cl, K, J)
    perms, vecs = translations(cl)
    psi = random_state(n, 3 + n)
    ctx = ftk.Context(cl, K, J, "fp64")
    for q in cl.momenta:
        chi = characters(vecs, q)
        reps, B = sector.basis(n, perms, chi)
        sec = ftk.Sector(ctx, perms, chi, n_slots=4)
        d, n_orb, got_reps = sec.info()
        assert d == len(reps) and np.array_equal(got_reps.astype(np.int64), reps)
        sec.project(psi, 0)
        assert rel(sec.get(0), B.conj().T @ psi) <= 1e-13
        rng = np.random.default_rng(d)
        v = rng.standard_normal(d) + 1j * rng.standard_normal(d)
        sec.set(1, v)
        sec.hv(1, 2)
        assert rel(sec.get(2), sector.block(H, B) @ v) <= 1e-12
        sec.close()
    ctx.close()


def test_sector_hv_n20_matrix_free(ftk):
    """20-site torus (2x5, 10 translations), a nonzero momentum: the sector
    H.v against embed -> full H (the oracle's C H.v) -> project."""
    cl = named(20)
    K, J = -1.0, 0.1
    perms, vecs = translations(cl)
    q = cl.momenta[3]
    chi = characters(vecs, q)
    reps, orbit = sector.representatives(20, perms, chi)
    ctx = ftk.Context(cl, K, J, "fp64")
    sec = ftk.Sector(ctx, perms, chi, n_slots=2)
    assert sec.dim == len(reps)
    rng = np.random.default_rng(20)
    v = rng.standard_normal(len(reps)) + 1j * rng.standard_normal(len(reps))
    sec.set(0, v)
    sec.hv(0, 1)
    want = sector.project(sparse.hv(cl, K, J, sector.embed(v, reps, orbit, perms, chi, 20)), reps, orbit, perms, chi)
    assert rel(sec.get(1), want) <= 1e-12
    sec.close()
    ctx.close()


def test_sector_green_vs_dense_resolvent(ftk):
    cl = named(12)
    K, J = -1.0, 0.1
    H = dense.hamiltonian(cl, K, J)
    perms, vecs = translations(cl)
    ctx = ftk.Context(cl, K, J, "fp64")
    z = np.linspace(-3, 3, 61) + 0.05j
    for qi in (0, 2):
        chi = characters(vecs, cl.momenta[qi])
        reps, B = sector.basis(12, perms, chi)
        Hk = sector.block(H, B)
        E, V = np.linalg.eigh(Hk)
        rng = np.random.default_rng(qi)
        lam = rng.standard_normal(len(reps)) + 1j * rng.standard_normal(len(reps))
        sec = ftk.Sector(ctx, perms, chi, n_slots=4)
        sec.set(0, lam)
        G, it = sec.green(0, z, tol=1e-12, max_iter=5000)
        c = V.conj().T @ lam
        want = np.array([np.sum(np.abs(c) ** 2 / (zz - E)) for zz in z])
        assert np.abs(G - want).max() <= 1e-9 * np.abs(want).max()
        # without reorthogonalisation Lanczos loses orthogonality in floating
        # point and may take more steps than the dimension; G still converges
        assert 0 < it <= 4 * len(reps)
        sec.close()
    ctx.close()


def test_sector_pipeline_vs_full_basis_estimator(ftk):
    """N = 12: the full random state split into the 6 momentum sectors; the
    mTPQ iteration in each (61 steps, shells every 20); merged statistics
    against the oracle's full-basis iteration; S^z_q from every sector Q to
    Q + q; Lanczos G per sector; merged G and the reweighted spectrum against
    the oracle's eigenbasis estimator on the full state (1e-8)."""
    cl = named(12)
    K, J, ell = -1.0, 0.1, 0.5
    n_steps, se = 61, 20
    psi0 = random_state(12, 99)
    perms, vecs = translations(cl)
    qi = 1
    q = cl.momenta[qi]
    omega = omega_grid(-2, 2, 128)
    eta = 0.05
    T = np.array([0.5, 1.0, 2.0])
    ctx = ftk.Context(cl, K, J, "fp64", max_rhs=1, n_saved=1)
    chis = [characters(vecs, Q) for Q in cl.momenta]
    n_sh = (n_steps + se - 1) // se
    secs = [ftk.Sector(ctx, perms, ch, n_slots=n_sh + 6) for ch in chis]
    # the sector of Q + q for each Q (characters multiply)
    dst = []
    for ch in chis:
        target = ch * characters(vecs, q)
        dst.append(int(np.argmin([np.abs(target - c2).max() for c2 in chis])))
    lognorm0, logq, us = [], [], []
    for s in secs:
        s.project(psi0, 0)
        u, lq, l0 = s.tpq(0, 1, ell, n_steps, se, 2)
        lognorm0.append(l0)
        logq.append(lq)
        us.append(u)
    steps = np.arange(0, n_steps, se)
    Gs = np.zeros((len(secs), n_sh, len(omega)), dtype=np.complex128)
    # per shell: sector shift origin E_k = N u_k of the merged statistics
    u_m, lq_m, _ = ftk.ftk_sector_combine(lognorm0, logq, us)
    _, ur, lqr, _ = sparse.tpq(cl, K, J, psi0, ell, n_steps, se)
    assert np.abs(u_m - ur).max() <= 1e-12
    assert np.abs(lq_m - lqr).max() <= 1e-11
    probe = n_sh + 2
    for si, s in enumerate(secs):
        for sh in range(n_sh):
            s.apply_sz(2 + sh, secs[dst[si]], probe, q)
            z = 12 * u_m[steps[sh]] + omega + 1j * eta
            G, _ = secs[dst[si]].green(probe, z, tol=1e-12, max_iter=5000)
            Gs[si, sh] = G
    u_c, lq_c, G = ftk.ftk_sector_combine(lognorm0, logq, us, steps, Gs)
    S, tr = ctx.spectrum_ex(G, T, u_c, lq_c, se, ell)
    for s in secs:
        s.close()
    ctx.close()
    dg = dense.Diag(cl, K, J)
    ref = dense.dense_estimator(dg, psi0, ell, n_steps, se, 2, q, omega, eta, T)
    assert rel(G.ravel(), ref["G"].ravel()) <= 1e-8
    assert rel(S, ref["S"]) <= 1e-8
    assert tr.tolist() == ref["trunc"].astype(int).tolist()


def test_sector_checks(ftk):
    cl = named(8)
    perms, vecs = translations(cl)
    ctx = ftk.Context(cl, -1.0, 0.1, "fp64")
    chi = characters(vecs, cl.momenta[1])
    bad_perm = perms.copy()
    bad_perm[1] = np.roll(bad_perm[1], 1)                 # not a translation: breaks bonds / closure
    for P, ch in ((bad_perm, chi), (perms, chi * np.exp(0.3j)), (perms[1:], chi[1:])):
        with pytest.raises(ftk.FtkError) as e:
            ftk.Sector(ctx, P, ch)
        assert e.value.status == ftk.FTK_EINVAL
    s0 = ftk.Sector(ctx, perms, characters(vecs, cl.momenta[0]), n_slots=4)
    s1 = ftk.Sector(ctx, perms, chi, n_slots=4)
    with pytest.raises(ftk.FtkError):
        s0.apply_sz(0, s1, 0, cl.momenta[2])              # the destination is not Q + q
    s0.close()
    s1.close()
    ctx.close()
