"""Pins of the oracle's Hamiltonian (Sec. V.A) against brute force, closed
forms and symmetries. CPU only."""
import itertools

import numpy as np
import pytest

from ftk_inputs import named, honeycomb, random_state
from oracle import dense, sparse

KJ = [(-1.0, 0.1), (-1.0, 0.0), (0.0, 1.0), (0.7, -0.3)]


@pytest.mark.parametrize("n", [2, 4, 6, 8, 12])
@pytest.mark.parametrize("K,J", KJ)
def test_matrix_free_equals_kronecker(n, K, J):
    """Brute force: bit-rule H v (sparse.c) == Kronecker-product H v."""
    if n == 12 and (K, J) != (-1.0, 0.1):
        pytest.skip("one N=12 case is enough")
    cl = named(n)
    h = dense.hamiltonian(cl, K, J)
    v = random_state(n, 7)
    out = sparse.hv(cl, K, J, v)
    ref = h @ v
    assert np.linalg.norm(out - ref) <= 1e-14 * np.linalg.norm(ref)


@pytest.mark.parametrize("n", [8, 12])
@pytest.mark.parametrize("K,J", KJ)
def test_trace_closed_forms(n, K, J):
    """Tr H = 0 and Tr H^2 / 2^N = n_bonds (K^2 + 2JK + 3J^2)/16 (no repeated pairs)."""
    cl = named(n)
    pairs = {tuple(sorted(b[:2])) for b in cl.bonds.tolist()}
    assert len(pairs) == cl.n_bonds
    h = dense.hamiltonian(cl, K, J)
    d = h.shape[0]
    assert abs(np.trace(h)) < 1e-12
    want = cl.n_bonds * (K * K + 2 * J * K + 3 * J * J) / 16
    assert abs(np.sum(h * h) / d - want) < 1e-12


@pytest.mark.parametrize("K,J", KJ)
def test_hermitian_and_real(K, J):
    """<u|Hv> = <Hu|v> and H conj(v) = conj(H v) (H real symmetric)."""
    cl = named(12)
    u = random_state(12, 1)
    v = random_state(12, 2)
    hu = sparse.hv(cl, K, J, u)
    hv = sparse.hv(cl, K, J, v)
    assert abs(np.vdot(u, hv) - np.vdot(hu, v)) < 1e-13
    assert np.abs(sparse.hv(cl, K, J, v.conj()) - hv.conj()).max() < 1e-15


def test_dimer_closed_form():
    """1x1 torus: all three bonds join A and B, H = (K + 3J) S_A.S_B:
    singlet -3(K+3J)/4, triplet (K+3J)/4 (threefold)."""
    cl = honeycomb((1, 1))
    K, J = -1.0, 0.3
    lam = K + 3 * J
    e = np.sort(np.linalg.eigvalsh(dense.hamiltonian(cl, K, J)))
    assert np.allclose(e, np.sort([-0.75 * lam, 0.25 * lam, 0.25 * lam, 0.25 * lam]), atol=1e-14)


def _sz_total(x, n):
    return sum(((x >> l) & 1) * 2 - 1 for l in range(n))


def test_heisenberg_conserves_total_sz():
    """K = 0: H maps an S^z_tot = m sector into itself, exact zeros elsewhere."""
    n = 12
    cl = named(n)
    d = 1 << n
    sz = np.array([_sz_total(x, n) for x in range(d)])
    v = random_state(n, 3)
    v[sz != 2] = 0
    out = sparse.hv(cl, 0.0, 1.0, v)
    assert np.all(out[sz != 2] == 0)
    assert np.linalg.norm(out[sz == 2]) > 0.1
    out_k = sparse.hv(cl, -1.0, 0.0, v)          # Kitaev terms break it
    assert np.linalg.norm(out_k[sz != 2]) > 0.1


def test_heisenberg_su2_multiplets():
    """K = 0: each degenerate eigenspace decomposes into full SU(2) multiplets:
    the multiplicity of S(S+1) inside it is a multiple of 2S+1."""
    n = 8
    cl = named(n)
    dg = dense.Diag(cl, 0.0, 1.0)
    s_tot = [sum(dense.site_op(n, l, dense.SPIN[a]) for l in range(n)).toarray() for a in range(3)]
    s2 = sum(s @ s for s in s_tot).real
    for s in s_tot:                       # [H, S_tot] = 0
        assert np.abs(dg.h @ s - s @ dg.h).max() < 1e-12
    e = dg.E
    i = 0
    while i < len(e):
        j = i
        while j < len(e) and e[j] - e[i] < 1e-9:
            j += 1
        sub = dg.V[:, i:j]
        ev = np.linalg.eigvalsh(sub.T @ s2 @ sub)
        svals = (-1 + np.sqrt(1 + 4 * ev)) / 2
        for sv in np.unique(np.round(svals * 2) / 2):
            cnt = int(np.sum(np.abs(svals - sv) < 1e-6))
            assert cnt % int(round(2 * sv + 1)) == 0
        i = j


def _hexagons(cl):
    adj = {i: [] for i in range(cl.n_sites)}
    for i, j, g in cl.bonds.tolist():
        adj[i].append((j, g))
        adj[j].append((i, g))
    found = set()
    for start in range(cl.n_sites):
        stack = [(start, [start])]
        while stack:
            node, path = stack.pop()
            if len(path) == 6:
                if any(nb == start for nb, _ in adj[node]):
                    found.add(frozenset(path))
                continue
            for nb, _ in adj[node]:
                if nb not in path:
                    stack.append((nb, path + [nb]))
    return [sorted(h) for h in found]


def test_kitaev_plaquettes_commute():
    """J = 0: the plaquette operators W_p = prod_{l in p} sigma^{gamma_out(l)}
    commute with H (Kitaev's conserved fluxes); J != 0 breaks this."""
    n = 12
    cl = named(n)
    hexes = _hexagons(cl)
    assert len(hexes) >= n // 2
    h0 = dense.hamiltonian_sparse(cl, -1.0, 0.0)
    h1 = dense.hamiltonian_sparse(cl, -1.0, 0.2)
    broken = 0
    for hx in hexes[: n // 2]:
        inside = set(hx)
        w = None
        for l in hx:
            outs = [g for i, j, g in cl.bonds.tolist()
                    if (i == l and j not in inside) or (j == l and i not in inside)]
            assert len(outs) == 1
            f = 2 * dense.site_op(n, l, dense.SPIN[outs[0]])
            w = f if w is None else w @ f
        assert abs(h0 @ w - w @ h0).max() < 1e-12
        broken += abs(h1 @ w - w @ h1).max() > 1e-3
    assert broken > 0


def test_ell_lower_bound_keeps_l_minus_h_positive():
    """The bond block h_b = J S_i.S_j + K S^g_i S^g_j has eigenvalues
    (J+K)/4 (x2), (J-K)/4, -(3J+K)/4, so l >= (1/N) sum_b lambda_max(h_b)
    guarantees l - H/N >= 0 (needed for positive R1 weights)."""
    for K, J in [(-1.0, 0.1), (-1.0, 0.2), (-1.0, -0.3)]:
        blk = (J * sum(np.kron(s, s) for s in dense.SPIN) + K * np.kron(dense.SZ, dense.SZ)).real
        ev = np.sort(np.linalg.eigvalsh(blk))
        assert np.allclose(ev, np.sort([(J + K) / 4, (J + K) / 4, (J - K) / 4, -(3 * J + K) / 4]))
        cl = named(8)
        lmin = cl.n_bonds * ev[-1] / cl.n_sites
        e = np.linalg.eigvalsh(dense.hamiltonian(cl, K, J))
        assert lmin - e.max() / cl.n_sites >= -1e-12


@pytest.mark.parametrize("n", [2, 8, 12])
@pytest.mark.parametrize("K,J", KJ)
def test_sampled_rows_equal_kronecker(n, K, J):
    """Brute force: the row-by-row product of oracle/rows.py (spin matrix
    elements per bond) == the Kronecker-product H v, on every row."""
    from oracle import rows
    cl = named(n)
    h = dense.hamiltonian_sparse(cl, K, J)
    v = random_state(n, 11)
    xs = np.arange(1 << n, dtype=np.int64)
    got = rows.hv_rows(cl, K, J, lambda idx: v[idx], xs)
    ref = h @ v
    assert np.linalg.norm(got - ref) <= 1e-14 * np.linalg.norm(ref)


def test_sampled_rows_of_a_bigger_cluster():
    """At N = 16 on random rows: the row formula against the matrix-free C
    product (two independent codings of the same matrix elements)."""
    from oracle import rows
    cl = named(16)
    v = random_state(16, 5)
    xs = np.random.default_rng(3).integers(0, 1 << 16, 512)
    got = rows.hv_rows(cl, -1.0, 0.05, lambda idx: v[idx], xs)
    ref = sparse.hv(cl, -1.0, 0.05, v)[xs]
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()
