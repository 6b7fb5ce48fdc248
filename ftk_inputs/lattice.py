"""Periodic honeycomb clusters: sites, positions, bonds and cluster momenta.

This module is an *input generator*: it builds the geometry that both the
CUDA path and the CPU oracle receive as input. It holds none of the method's
arithmetic (no Hamiltonian matrix elements, no spin algebra).

Geometry (the paper's Sec. V, Fig. 'fig_honeycomb_18_24' and the bond
directions listed in its caption): x, y and z bonds lie along -60, +60 and
0 degree lines. Site A of the cell at R sits at R, site B at R + d_z.

    d_z = (1, 0),  d_x = (-1/2, sqrt(3)/2),  d_y = (-1/2, -sqrt(3)/2)
    a_1 = d_z - d_x,  a_2 = d_z - d_y

    z-bond: A(R) - B(R);  x-bond: A(R) - B(R - a_1);  y-bond: A(R) - B(R - a_2)

A cluster is the torus Z^2 / M Z^2 of unit cells, where the rows of the
integer matrix M are the supercell vectors in units of (a_1, a_2). An
L1 x L2 torus has M = diag(L1, L2). The figure in the paper gives the
shapes of its 12/18/24-site clusters only graphically, so the tori here are
the L1 x L2 (or tilted) shapes named by the workloads.

Site numbering: cell c -> A = 2c, B = 2c + 1. Positions R_l are the real
site coordinates (not the cell origin), as the paper specifies for S_Q
(Sec. V, below Eq. 'SQomega_TPS').
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA_X, GAMMA_Y, GAMMA_Z = 0, 1, 2

_S3 = math.sqrt(3.0)
D_Z = np.array([1.0, 0.0])
D_X = np.array([-0.5, _S3 / 2])
D_Y = np.array([-0.5, -_S3 / 2])
A1 = D_Z - D_X
A2 = D_Z - D_Y


def _reciprocal():
    a = np.stack([A1, A2])            # rows a_i
    b = 2 * math.pi * np.linalg.inv(a).T   # rows b_i with a_i . b_j = 2 pi delta_ij
    return b[0], b[1]


B1, B2 = _reciprocal()


@dataclass
class Cluster:
    """A periodic honeycomb cluster.

    n_sites: N; pos: float64 [N, 2]; bonds: int32 [n_bonds, 3] rows (i, j, gamma);
    momenta: float64 [N/2, 2] cluster momenta inside the first Brillouin zone;
    momentum_index: int [N/2, 2] the integer labels (k1, k2) * det(M) of each momentum;
    supercell: the integer matrix M.
    """
    n_sites: int
    pos: np.ndarray
    bonds: np.ndarray
    momenta: np.ndarray
    momentum_index: np.ndarray
    supercell: np.ndarray
    name: str = ""
    perm: np.ndarray | None = field(default=None)

    @property
    def n_bonds(self) -> int:
        return int(self.bonds.shape[0])

    @property
    def dim(self) -> int:
        return 1 << self.n_sites


def _cells(m: np.ndarray):
    """Integer representatives of Z^2 / M Z^2 and a reducer to them."""
    det = int(round(np.linalg.det(m)))
    if det <= 0:
        raise ValueError("supercell matrix must have positive determinant")
    adj = np.array([[m[1, 1], -m[0, 1]], [-m[1, 0], m[0, 0]]], dtype=np.int64)

    def reduce(n):
        n = np.asarray(n, dtype=np.int64)
        f = n @ adj                         # = det * fractional coordinates
        u = np.floor_divide(f, det)
        return tuple(int(v) for v in (n - u @ m))

    reps = []
    seen = set()
    lo0 = min(0, m[0, 0], m[1, 0], m[0, 0] + m[1, 0])
    hi0 = max(0, m[0, 0], m[1, 0], m[0, 0] + m[1, 0])
    lo1 = min(0, m[0, 1], m[1, 1], m[0, 1] + m[1, 1])
    hi1 = max(0, m[0, 1], m[1, 1], m[0, 1] + m[1, 1])
    for n2 in range(lo1, hi1 + 1):
        for n1 in range(lo0, hi0 + 1):
            r = reduce((n1, n2))
            if r not in seen:
                seen.add(r)
                reps.append(r)
    if len(reps) != det:
        raise RuntimeError("cell enumeration failed")
    # deterministic order: by (n2, n1)
    reps.sort(key=lambda t: (t[1], t[0]))
    return reps, reduce, det


def _momenta(m: np.ndarray):
    """Cluster momenta Q with Q . T_i in 2 pi Z, folded into the first BZ.

    Q = k1 b1 + k2 b2 with M (k1, k2)^T integer. Among the images Q + G the
    one of smallest |Q + G| is kept (Wigner-Seitz cell around Gamma); ties
    (within 1e-9) go to the lexicographically smallest (g1, g2).
    """
    det = int(round(np.linalg.det(m)))
    minv_det = np.array([[m[1, 1], -m[0, 1]], [-m[1, 0], m[0, 0]]], dtype=np.int64)
    ks = set()
    for n1 in range(det):
        for n2 in range(det):
            kd = minv_det @ np.array([n1, n2], dtype=np.int64)   # det * k
            ks.add((int(kd[0] % det), int(kd[1] % det)))
    ks = sorted(ks)
    if len(ks) != det:
        raise RuntimeError("momentum enumeration failed")
    qs, idx = [], []
    for k1d, k2d in ks:
        best = None
        for g1 in range(-3, 4):
            for g2 in range(-3, 4):
                q = (k1d / det + g1) * B1 + (k2d / det + g2) * B2
                n2 = float(q @ q)
                key = (round(n2, 9), g1, g2)
                if best is None or key < best[0]:
                    best = (key, q)
        qs.append(best[1])
        idx.append((k1d, k2d))
    return np.array(qs), np.array(idx, dtype=np.int64)


def honeycomb(supercell, name: str = "") -> Cluster:
    """Build the periodic honeycomb cluster for supercell matrix M (2x2 ints)
    or for a pair (L1, L2) meaning M = diag(L1, L2)."""
    if len(np.shape(supercell)) == 1:
        l1, l2 = supercell
        m = np.array([[l1, 0], [0, l2]], dtype=np.int64)
    else:
        m = np.array(supercell, dtype=np.int64)
    reps, reduce, det = _cells(m)
    index = {r: c for c, r in enumerate(reps)}
    n_sites = 2 * det
    pos = np.zeros((n_sites, 2))
    bonds = []
    for c, (n1, n2) in enumerate(reps):
        r = n1 * A1 + n2 * A2
        pos[2 * c] = r
        pos[2 * c + 1] = r + D_Z
    for c, (n1, n2) in enumerate(reps):
        a = 2 * c
        bonds.append((a, 2 * index[reduce((n1, n2))] + 1, GAMMA_Z))
        bonds.append((a, 2 * index[reduce((n1 - 1, n2))] + 1, GAMMA_X))
        bonds.append((a, 2 * index[reduce((n1, n2 - 1))] + 1, GAMMA_Y))
    bonds = np.array(bonds, dtype=np.int32)
    qs, qidx = _momenta(m)
    return Cluster(n_sites, pos, bonds, qs, qidx, m, name or f"honeycomb{n_sites}")


def relabel(cl: Cluster, perm) -> Cluster:
    """Return the same cluster with site l renamed perm[l] (a bit permutation
    of the Fock basis). Positions move with their sites."""
    perm = np.asarray(perm, dtype=np.int64)
    n = cl.n_sites
    if sorted(perm.tolist()) != list(range(n)):
        raise ValueError("not a permutation")
    pos = np.zeros_like(cl.pos)
    pos[perm] = cl.pos
    bonds = cl.bonds.copy()
    bonds[:, 0] = perm[cl.bonds[:, 0]]
    bonds[:, 1] = perm[cl.bonds[:, 1]]
    return Cluster(n, pos, bonds, cl.momenta.copy(), cl.momentum_index.copy(),
                   cl.supercell.copy(), cl.name, perm)


def translations(cl: Cluster):
    """The translation group of the torus as site permutations.

    Returns (perms int32 [n_cells, N], vectors float64 [n_cells, 2]): element g
    moves site l to site perms[g, l], the site at R_l + a_g modulo the
    supercell (a_g = vectors[g], a lattice vector); element 0 is the
    identity. Works from the positions, so it holds for relabelled clusters
    too. Geometry only: a momentum sector is chosen by the caller through
    the characters exp(-i Q . a_g)."""
    m = cl.supercell
    reps, reduce, det = _cells(m)
    a = np.stack([A1, A2])                 # rows a_1, a_2
    ainv = np.linalg.inv(a)
    n = cl.n_sites
    key = {}
    for l in range(n):
        for sub, off in ((0, np.zeros(2)), (1, D_Z)):
            f = (cl.pos[l] - off) @ ainv
            if np.allclose(f, np.round(f), atol=1e-9):
                cell = reduce(tuple(int(v) for v in np.round(f)))
                key[(sub, cell)] = l
                break
        else:
            raise RuntimeError("site position is not on the honeycomb lattice")
    site_key = {l: k for k, l in key.items()}
    cells = sorted(reps, key=lambda t: (t != (0, 0), t[1], t[0]))   # identity first
    perms, vecs = [], []
    for t1, t2 in cells:
        pm = np.zeros(n, dtype=np.int32)
        for l in range(n):
            sub, (n1, n2) = site_key[l]
            pm[l] = key[(sub, reduce((n1 + t1, n2 + t2)))]
        perms.append(pm)
        vecs.append(t1 * A1 + t2 * A2)
    return np.array(perms, dtype=np.int32), np.array(vecs)


def characters(vectors, q):
    """exp(-i q . a_g) for the translation vectors a_g (the sector of momentum q)."""
    return np.exp(-1j * (np.asarray(vectors) @ np.asarray(q, dtype=np.float64)))


# Named clusters used by the workloads (cells x 2 sites).
NAMED = {
    2: (1, 1),
    4: (1, 2),
    6: (1, 3),
    8: (2, 2),
    10: (1, 5),
    12: (2, 3),
    14: (1, 7),
    16: (2, 4),
    20: (2, 5),
    18: (3, 3),
    24: (3, 4),
    26: [[3, 1], [-1, 4]],   # 13 cells: tilted, avoids the 1 x 13 double bonds
    28: (2, 7),
    30: (3, 5),
}


def named(n_sites: int) -> Cluster:
    return honeycomb(NAMED[n_sites], f"honeycomb{n_sites}")
