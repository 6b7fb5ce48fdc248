"""Pins of oracle/sector.py (momentum sectors of the translation group),
against the dense Kronecker-product H and LAPACK: the sector basis is
orthonormal, each sector is an invariant subspace of H, the sector spectra
together are the spectrum of H, the sectors partition the basis, S^z_q maps
sector Q to sector Q + q, and the matrix-free project / embed equal B^dag, B.
CPU only."""
import numpy as np
import pytest

from ftk_inputs import named, translations, characters
from oracle import dense, sector, sparse


@pytest.mark.parametrize("n", [8, 12])
def test_sectors_partition_and_reproduce_the_spectrum(n):
    cl = named(n)
    K, J = -1.0, 0.1
    H = dense.hamiltonian(cl, K, J)
    perms, vecs = translations(cl)
    E_all, dims = [], 0
    for q in cl.momenta:
        chi = characters(vecs, q)
        reps, B = sector.basis(n, perms, chi)
        dims += len(reps)
        assert np.abs(B.conj().T @ B - np.eye(len(reps))).max() <= 1e-12
        Hk = sector.block(H, B)
        assert np.abs(Hk - Hk.conj().T).max() <= 1e-12
        assert np.abs(H @ B - B @ Hk).max() <= 1e-12       # invariant subspace
        E_all.append(np.linalg.eigvalsh(Hk))
    assert dims == 1 << n
    E = np.sort(np.concatenate(E_all))
    assert np.abs(E - np.linalg.eigvalsh(H)).max() <= 1e-10


def test_sz_q_maps_sector_q_to_q_plus_k():
    """lambda = S^z_k psi for psi in sector Q lies in sector Q + k (the
    character multiplied by exp(-i k.a_g))."""
    cl = named(12)
    perms, vecs = translations(cl)
    rng = np.random.default_rng(4)
    for a, b in [(0, 1), (2, 3), (4, 5)]:
        Q, k = cl.momenta[a], cl.momenta[b]
        chi_q = characters(vecs, Q)
        reps, B = sector.basis(12, perms, chi_q)
        psi = B @ (rng.standard_normal(len(reps)) + 1j * rng.standard_normal(len(reps)))
        lam = sparse.apply_op(cl, 2, k, psi)
        chi_qk = chi_q * characters(vecs, k)
        _, B2 = sector.basis(12, perms, chi_qk)
        assert np.linalg.norm(lam - B2 @ (B2.conj().T @ lam)) <= 1e-12 * np.linalg.norm(lam)


def test_matrix_free_project_and_embed():
    cl = named(12)
    perms, vecs = translations(cl)
    rng = np.random.default_rng(8)
    psi = rng.standard_normal(1 << 12) + 1j * rng.standard_normal(1 << 12)
    for q in cl.momenta[:3]:
        chi = characters(vecs, q)
        reps, orbit = sector.representatives(12, perms, chi)
        _, B = sector.basis(12, perms, chi)
        assert np.abs(sector.project(psi, reps, orbit, perms, chi) - B.conj().T @ psi).max() <= 1e-12
        v = rng.standard_normal(len(reps)) + 1j * rng.standard_normal(len(reps))
        assert np.abs(sector.embed(v, reps, orbit, perms, chi, 12) - B @ v).max() <= 1e-12
