"""Continuous batching on the GPU: jobs of different cluster sizes,
couplings, momenta, eta, temperatures and precisions (FP64, FP32, mixed,
double-float) run concurrently on their own streams; each result equals the
same job run alone, and one job is checked against the oracle's eigenbasis
estimator. GPU only."""
import numpy as np
import pytest

from ftk_inputs import named, omega_grid
from oracle import dense, sparse

pytestmark = pytest.mark.gpu


def _specs(serve):
    return [
        serve.JobSpec(n_sites=8, K=-1.0, J=0.1, seed=3, n_steps=31, save_every=10, probes=[(2, 1), (0, 2)],
                      omega=(-2, 2, 64), eta=0.05, temps=[0.3, 1.0], tol=1e-10, max_iter=3000, block=4),
        serve.JobSpec(n_sites=10, K=-1.0, J=-0.2, seed=5, n_steps=21, save_every=10, probes=[(1, 0)],
                      omega=(-3, 3, 100), eta=0.1, temps=[0.5], tol=1e-8, max_iter=3000, block=2),
        serve.JobSpec(n_sites=12, K=-1.0, J=0.2, seed=9, n_steps=21, save_every=20, probes=[(2, 3), (1, 1)],
                      omega=(-2, 2, 128), eta=0.1, temps=[0.4, 2.0], tol=1e-6, max_iter=3000, block=4,
                      precision="fp32"),
        serve.JobSpec(n_sites=12, K=-1.0, J=0.0, seed=11, n_steps=11, save_every=10, probes=[(2, 2)],
                      omega=(-2, 2, 64), eta=0.08, temps=[1.0], tol=1e-8, max_iter=3000, block=2,
                      precision="mixed"),
        serve.JobSpec(n_sites=10, K=-1.0, J=0.05, seed=13, n_steps=21, save_every=20, probes=[(2, 1), (0, 1)],
                      omega=(-3, 3, 128), eta=0.02, temps=[0.2, 1.0], tol=1e-9, max_iter=4000, block=4,
                      precision="df"),
    ]


def test_alone_equals_mixed_and_matches_oracle():
    from paper_1802_02854_gb300 import build
    build.build()
    from paper_1802_02854_gb300 import serve

    specs = _specs(serve)
    alone = []
    for sp in specs:
        srv = serve.Server(max_slots=1)
        alone.append(srv.result(srv.submit(sp), timeout=600))
        srv.close()
    srv = serve.Server(max_slots=4)
    ids = [srv.submit(sp) for sp in specs]
    mixed = [srv.result(j, timeout=600) for j in ids]
    st = srv.stats()
    srv.close()
    assert st["peak_running"] >= 2 and st["latency_p99_s"] >= st["latency_p50_s"] > 0
    for a, m in zip(alone, mixed):
        assert a.status == "ok" and m.status == "ok", (a.status, m.status)
        for key in a.spectra:
            sa, sm = a.spectra[key], m.spectra[key]
            assert np.linalg.norm(sa - sm) <= 1e-12 * np.linalg.norm(sa)
    # job 0 against the oracle's estimator (same seeded Philox state)
    sp = specs[0]
    cl = named(8)
    psi0 = sparse.gaussian_state(8, sp.seed, sp.sample)
    dg = dense.Diag(cl, sp.K, sp.J)
    om = omega_grid(*sp.omega)
    for (g, qi), S in alone[0].spectra.items():
        ref = dense.dense_estimator(dg, psi0, 0.5, sp.n_steps, sp.save_every, g, cl.momenta[qi], om, sp.eta,
                                    sp.temps)
        assert np.linalg.norm(S - ref["S"]) <= 1e-8 * np.linalg.norm(ref["S"])


@pytest.mark.parametrize("prec", ["fp64", "df"])
def test_packed_jobs_equal_alone(prec):
    """Three jobs on the same 12-site Hamiltonian (different seeds, probes and
    temperatures) waiting together are packed into one blocked solve; each
    job's spectra equal the job run alone (its own context and block) to 1e-9
    (both solved to tol 1e-11; the block width changes the H.V plan, so the
    rounding differs)."""
    from paper_1802_02854_gb300 import build
    build.build()
    from paper_1802_02854_gb300 import serve

    def job(seed, probes, temps):
        return serve.JobSpec(n_sites=12, K=-1.0, J=0.1, seed=seed, n_steps=41, save_every=20, probes=probes,
                             omega=(-2, 2, 96), eta=0.05, temps=temps, tol=1e-11, max_iter=5000, block=4,
                             precision=prec)

    specs = [job(21, [(2, 1)], [0.5, 1.0]), job(22, [(0, 2), (2, 3)], [0.7]), job(23, [(1, 4)], [0.4, 2.0])]
    alone = []
    for sp in specs:
        srv = serve.Server(max_slots=1)
        alone.append(srv.result(srv.submit(sp), timeout=600))
        srv.close()
    srv = serve.Server(max_slots=1, pack_rhs=32)
    blocker = srv.submit(serve.JobSpec(n_sites=10, J=0.2, seed=1, n_steps=21, omega=(-2, 2, 64), eta=0.1,
                                       tol=1e-8, temps=[1.0]))
    ids = [srv.submit(sp) for sp in specs]
    packed = [srv.result(j, timeout=600) for j in ids]
    srv.result(blocker, timeout=600)
    srv.close()
    assert srv.packs and sorted(srv.packs[0]) == ids
    for a, m in zip(alone, packed):
        assert a.status == "ok" and m.status == "ok", (a.status, m.status)
        for key in a.spectra:
            assert np.linalg.norm(a.spectra[key] - m.spectra[key]) <= 1e-9 * np.linalg.norm(a.spectra[key])
            assert a.trunc[key].tolist() == m.trunc[key].tolist()


def test_large_cluster_jobs():
    """The serving configuration's larger clusters through the server: a
    26-site double-float job and a 30-site job (2^30 amplitudes) in the mixed
    mode (FP32 H.v, double-float residuals; the FP32 mode's residual stalls
    above 1e-3 on this cluster's infinite-temperature shell), admitted by
    footprint and run concurrently. No oracle solve fits these sizes; the
    Green's functions must be those of a Hermitian H with eta > 0 (Im G < 0
    at every shift; -Im G is eta |(z - H)^-1 lambda|^2) and the reweighted
    spectra non-negative and finite."""
    import torch
    from paper_1802_02854_gb300 import build
    build.build()
    from paper_1802_02854_gb300 import serve

    torch.cuda.empty_cache()   # the server's budget is 90 % of the memory free now
    specs = [serve.JobSpec(n_sites=26, K=-1.0, J=0.1, seed=7, n_steps=21, save_every=20, probes=[(2, 1)],
                           omega=(-3, 3, 48), eta=0.2, temps=[2.0, 4.0], tol=1e-4, max_iter=3000, block=1,
                           precision="df"),
             serve.JobSpec(n_sites=30, K=-1.0, J=-0.1, seed=8, n_steps=21, save_every=20, probes=[(2, 2)],
                           omega=(-3, 3, 32), eta=0.2, temps=[2.0, 4.0], tol=1e-4, max_iter=3000, block=1,
                           precision="mixed")]
    srv = serve.Server(max_slots=2)
    ids = [srv.submit(sp) for sp in specs]
    res = [srv.result(j, timeout=1200) for j in ids]
    st = srv.stats()
    srv.close()
    assert st["peak_mem_bytes"] >= max(sp.footprint() for sp in specs)
    for sp, r in zip(specs, res):
        assert r.status == "ok", r.status
        for key, G in r.G.items():
            G = np.asarray(G)
            assert np.isfinite(G).all()
            assert (G.imag < 0).all(), (sp.n_sites, G.imag.max())
            S = np.asarray(r.spectra[key])
            assert np.isfinite(S).all() and S.min() >= -1e-9 * np.abs(S).max()
