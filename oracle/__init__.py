"""The oracle: a plain, slow, obviously correct CPU implementation of the
FTKomega hot path (arXiv:1802.02854), in FP64.

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference legs may import, call, link or execute anything
under oracle/. The product package never does, and the oracle never imports
the product package; the two share only the seeded input generators in
ftk_inputs/.

Parts:
  dense.py    Kronecker-product H, canonical spectrum (Eq. chiAB), and the
              same estimator the CUDA path computes, evaluated exactly in the
              eigenbasis (N <= 12).
  sparse.c    matrix-free H v, mTPQ, S^gamma_q, textbook shifted COCG
              (projected and unprojected), canonical sum, Philox4x32-10.
  reweight.py reading R1: mTPQ shells to temperatures via Eq. B1.
  ctpq.py     cTPQ state at inverse temperature beta: the Taylor series of
              Eq. B1 in M_d steps (Appendix A).
  filter.py   contour filter operators, equi-energy shells, their
              probability distribution and Green's function (Sec. II.C-D).
  cocg3.py    shifted COCG in the three-term (residual-only) form of the
              CUDA path, with optional seed switching.
  sector.py   momentum sectors of the translation group: the sector basis
              from its definition, the sector block of H, projection and
              embedding.
  rows.py     sampled rows of H v from the spin matrix elements, for
              clusters (26, 30 sites) where no full product fits a test.

Every function is pinned by -m "not gpu" tests (tests/test_oracle_*.py)
against closed forms, brute force, invariants and published test vectors.
"""
