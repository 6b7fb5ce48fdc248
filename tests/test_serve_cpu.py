"""Scheduler of the spectrum server on the CPU: admission by footprint,
concurrency up to the slot count, skip-ahead without starvation, failures
isolated, latency statistics. The runner is a fake (no GPU)."""
import threading
import time

import pytest

from paper_1802_02854_gb300.serve import JobSpec, Server


class FakeRunner:
    def __init__(self, delay=0.05, fail_on=()):
        self.delay = delay
        self.fail_on = set(fail_on)
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0
        self.order = []

    def __call__(self, spec):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
            self.order.append(spec.seed)
        try:
            time.sleep(self.delay)
            if spec.seed in self.fail_on:
                raise RuntimeError("planted failure")
            return {"status": "ok", "spectra": {(2, 1): [[float(spec.seed)]]}}
        finally:
            with self.lock:
                self.active -= 1


def fp(spec):
    return spec.n_sites * 100   # bytes: proportional to the cluster size


def test_slots_bound_concurrency_and_all_finish():
    run = FakeRunner()
    srv = Server(max_slots=3, mem_budget=10_000, runner=run, footprint=fp)
    ids = [srv.submit(JobSpec(n_sites=8, seed=s)) for s in range(10)]
    res = [srv.result(i, timeout=30) for i in ids]
    srv.close()
    assert all(r.status == "ok" for r in res)
    assert run.max_active == 3 and srv.stats()["peak_running"] == 3
    assert [r.spectra[(2, 1)][0][0] for r in res] == list(range(10))


def test_memory_budget_limits_admission():
    run = FakeRunner(delay=0.05)
    srv = Server(max_slots=8, mem_budget=2500, runner=run, footprint=fp)   # two 12-site jobs fit
    ids = [srv.submit(JobSpec(n_sites=12, seed=s)) for s in range(6)]
    [srv.result(i, timeout=30) for i in ids]
    srv.close()
    assert run.max_active == 2
    assert srv.peak_mem <= 2500
    assert all(used <= 2500 for _, _, used in srv.admission_log)


def test_small_jobs_pass_a_blocked_large_one_without_starving_it():
    run = FakeRunner(delay=0.1)
    srv = Server(max_slots=4, mem_budget=3000, runner=run, footprint=fp, max_skips=2)
    a = srv.submit(JobSpec(n_sites=20, seed=0))    # 2000 B, runs
    b = srv.submit(JobSpec(n_sites=20, seed=1))    # does not fit beside a
    small = [srv.submit(JobSpec(n_sites=4, seed=10 + k)) for k in range(6)]
    res = {j: srv.result(j, timeout=30) for j in [a, b] + small}
    srv.close()
    assert all(r.status == "ok" for r in res.values())
    # some small job started before b (skip-ahead), but b was not passed over
    # by all of them (bounded skips)
    assert min(res[s].start for s in small) < res[b].start
    assert res[b].start <= max(res[s].start for s in small)


def test_oversized_job_is_rejected_and_failures_are_isolated():
    run = FakeRunner(fail_on={3})
    srv = Server(max_slots=2, mem_budget=1000, runner=run, footprint=fp)
    big = srv.submit(JobSpec(n_sites=30, seed=9))   # 3000 B > budget
    ids = [srv.submit(JobSpec(n_sites=4, seed=s)) for s in range(5)]
    res = [srv.result(i, timeout=30) for i in ids]
    srv.close()
    assert srv.result(big).status.startswith("error: footprint")
    assert res[3].status.startswith("error: RuntimeError")
    assert [r.status for k, r in enumerate(res) if k != 3] == ["ok"] * 4
    st = srv.stats()
    assert st["jobs"] == 4 and st["failed"] == 2


def test_latency_percentiles():
    run = FakeRunner(delay=0.02)
    srv = Server(max_slots=1, mem_budget=10_000, runner=run, footprint=fp)
    ids = [srv.submit(JobSpec(n_sites=4, seed=s)) for s in range(5)]
    res = [srv.result(i, timeout=30) for i in ids]
    srv.close()
    st = srv.stats()
    lat = sorted(r.latency for r in res)
    assert st["latency_p50_s"] == pytest.approx(lat[2])
    assert lat[0] <= st["latency_p99_s"] <= lat[-1] + 1e-12
    assert all(r.queue_wait >= 0 and r.finish >= r.start for r in res)


def test_submit_after_close_raises():
    srv = Server(max_slots=1, mem_budget=100, runner=FakeRunner(), footprint=fp)
    srv.close()
    with pytest.raises(RuntimeError):
        srv.submit(JobSpec(n_sites=4))


def test_poisson_stream_is_seeded_and_in_range():
    from paper_1802_02854_gb300 import serve
    a = serve.poisson_stream(30, seed=7, rate=3.0)
    b = serve.poisson_stream(30, seed=7, rate=3.0)
    assert [(t, s.n_sites, s.J, s.precision) for t, s in a] == [(t, s.n_sites, s.J, s.precision) for t, s in b]
    ts = [t for t, _ in a]
    assert all(t1 > t0 for t0, t1 in zip(ts, ts[1:]))
    for _, s in a:
        assert s.n_sites in (12, 16, 18, 20) and -0.3 <= s.J <= 0.3 and s.eta in (0.01, 0.02)
        assert 16 <= len(s.temps) <= 64 and s.omega[2] in (256, 512, 1024)
        assert all(0 <= g <= 2 and 0 <= q < s.n_sites // 2 for g, q in s.probes)
        assert s.precision in ("fp64", "df")


def test_compatible_jobs_are_packed():
    """pack_rhs: a job being admitted takes waiting jobs with the same pack key
    (same Hamiltonian, precision, shifts, eta, tolerance) along, up to the
    right-hand-side limit; other jobs run alone; every job gets its own result."""
    calls = []

    def pack_runner(specs):
        calls.append([s.seed for s in specs])
        time.sleep(0.02)
        return [{"status": "ok", "spectra": {(2, 1): [[float(s.seed)]]}} for s in specs]

    run = FakeRunner(delay=0.2)
    srv = Server(max_slots=1, mem_budget=100_000, runner=run, footprint=fp, pack_rhs=8, pack_runner=pack_runner)
    blocker = srv.submit(JobSpec(n_sites=8, J=0.3, seed=100))          # occupies the slot meanwhile
    same = [srv.submit(JobSpec(n_sites=8, J=0.1, seed=s, probes=[(2, s % 4)], n_steps=41)) for s in range(5)]
    other = srv.submit(JobSpec(n_sites=8, J=0.2, seed=50))              # another Hamiltonian
    res = {j: srv.result(j, timeout=30) for j in [blocker, other] + same}
    srv.close()
    assert all(r.status == "ok" for r in res.values())
    # 3 shells x 1 probe = 3 right-hand sides each: two jobs per pack of <= 8
    assert calls == [[0, 1], [2, 3], [4]] or calls == [[0, 1], [2, 3]]
    assert [res[j].spectra[(2, 1)][0][0] for j in same] == [0.0, 1.0, 2.0, 3.0, 4.0]
    assert len(srv.packs) >= 2 and run.order[0] == 100 and 50 in run.order
