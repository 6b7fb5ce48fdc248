"""Continuous-batching server for FTKomega spectrum jobs on one GPU.

Jobs (cluster size N, couplings K and J, probes S^gamma_q, eta, shift grid,
temperature grid, precision) arrive at any time. A scheduler thread admits a
waiting job as soon as a slot is free and its device footprint (the
ftk_footprint workspace plus a fixed allowance for the context's small
buffers) fits in the memory budget; a job that does not fit lets smaller
jobs behind it go first (no job is passed over more than `max_skips`
times). Each admitted job runs on its own CUDA stream in its own worker
thread with its own context, so the kernels of concurrent jobs overlap on the
device and later arrivals are admitted as earlier ones finish. A job: mTPQ
steps from its seeded state (Appendix A), the probes S^gamma_q on every saved
shell (Sec. V), blocked shifted COCG (probes packed in blocks of `block`
right-hand sides), reweighting to the temperature grid (Eq. B1, reading R1).

Every number a job returns comes from the CUDA library; the server only
schedules. A job's arithmetic does not depend on what else runs (own context
and stream, deterministic reductions), so its result is the same alone and in
the mix. The scheduler logic takes its runner and footprint functions as
arguments, so it is testable without a GPU.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

CTX_OVERHEAD_BYTES = 64 << 20   # small device buffers of a context + allocator slack


@dataclass
class JobSpec:
    """One spectrum job; probes are (gamma, momentum index) pairs, one spectrum each."""
    n_sites: int
    K: float = -1.0
    J: float = 0.1
    seed: int = 1
    sample: int = 0
    ell: float | None = None          # None: max(0.5, l_min)
    n_steps: int = 21
    save_every: int = 20
    probes: list = field(default_factory=lambda: [(2, 1)])
    omega: tuple = (-3.0, 3.0, 256)   # (min, max, count), endpoints included
    eta: float = 0.02
    temps: list = field(default_factory=lambda: [0.1, 0.5, 1.0])
    precision: str = "fp64"           # "fp64", "fp32", "mixed" or "df"
    tol: float = 1e-4
    max_iter: int = 10000
    block: int = 4
    cluster: object = None            # prebuilt cluster (default: the named honeycomb torus)

    @property
    def n_shells(self):
        return (self.n_steps + self.save_every - 1) // self.save_every

    def footprint(self):
        from . import PRECISIONS, ftk_footprint
        return ftk_footprint(self.n_sites, self.n_shells, self.block, PRECISIONS[self.precision]) + CTX_OVERHEAD_BYTES

    @property
    def n_rhs(self):
        """Right-hand sides of the job: every probe on every saved shell."""
        return len(self.probes) * self.n_shells

    def pack_key(self):
        """Jobs with equal keys can share one blocked solve: the same cluster
        and Hamiltonian, precision, shift grid, eta and stopping rule (the
        seeds, probes and temperatures may differ)."""
        cl = ("named", self.n_sites) if self.cluster is None else ("cluster", id(self.cluster))
        return (cl, float(self.K), float(self.J), self.ell, self.precision, tuple(self.omega), float(self.eta),
                float(self.tol), int(self.max_iter))


@dataclass
class JobResult:
    job_id: int
    status: str                       # "ok", "noconv", "error: ..."
    spectra: dict = field(default_factory=dict)   # probe -> S [n_T, n_omega]
    G: dict = field(default_factory=dict)         # probe -> G [n_shell, n_omega]
    iters: dict = field(default_factory=dict)     # probe -> iterations per shell
    trunc: dict = field(default_factory=dict)     # probe -> truncation flags per T
    arrival: float = 0.0
    start: float = 0.0
    finish: float = 0.0

    @property
    def latency(self):
        return self.finish - self.arrival

    @property
    def queue_wait(self):
        return self.start - self.arrival


def ell_for(cl, K, J, ell=None):
    """l of the job: max(0.5, l_min) unless given; l_min = (1/N) sum_b lambda_max(h_b)
    with the bond spectrum (J+K)/4 (twice), (J-K)/4, -(3J+K)/4."""
    lmax = max((J + K) / 4, (J - K) / 4, -(3 * J + K) / 4)
    lmin = len(cl.bonds) * lmax / cl.n_sites
    return max(0.5, lmin) if ell is None else ell


def run_job(spec: JobSpec, stream=None):
    """Run one job to completion through the C-ABI (blocking). Returns a
    dict with spectra, G, iters, trunc and status."""
    import torch

    from . import FTK_ENOCONV, Context
    from ftk_inputs import named, omega_grid

    cl = spec.cluster if spec.cluster is not None else named(spec.n_sites)
    omega = omega_grid(*spec.omega)
    temps = np.asarray(spec.temps, dtype=np.float64)
    stream = stream if stream is not None else torch.cuda.Stream()
    ctx = Context(cl, spec.K, spec.J, spec.precision, max_rhs=spec.block, n_saved=spec.n_shells, stream=stream)
    try:
        ctx.tpq_init(spec.seed, spec.sample, ell_for(cl, spec.K, spec.J, spec.ell))
        ctx.tpq_step(spec.n_steps, spec.save_every)
        steps, _ = ctx.shells()
        n_sh = len(steps)
        # every (probe, shell) is one right-hand side; pack them in blocks
        rhs = [(p, s) for p in range(len(spec.probes)) for s in range(n_sh)]
        G = {p: np.zeros((n_sh, len(omega)), dtype=np.complex128) for p in range(len(spec.probes))}
        iters = {p: np.zeros(n_sh, dtype=np.int64) for p in range(len(spec.probes))}
        status = "ok"
        for b0 in range(0, len(rhs), spec.block):
            blk = rhs[b0:b0 + spec.block]
            for slot, (p, s) in enumerate(blk):
                g, qi = spec.probes[p]
                ctx.apply_op(s, g, cl.momenta[qi], slot)
            Gb, it, st = ctx.shifted_cocg(list(range(len(blk))), omega, spec.eta, tol=spec.tol,
                                          max_iter=spec.max_iter, allow_noconv=True)
            if st == FTK_ENOCONV:
                status = "noconv"
            for slot, (p, s) in enumerate(blk):
                G[p][s] = Gb[slot]
                iters[p][s] = it[slot]
        spectra, trunc = {}, {}
        for p, probe in enumerate(spec.probes):
            S, tr = ctx.spectrum(G[p], temps)
            spectra[tuple(probe)] = S
            trunc[tuple(probe)] = tr
        return {"status": status, "spectra": spectra, "G": {tuple(spec.probes[p]): G[p] for p in G},
                "iters": {tuple(spec.probes[p]): iters[p] for p in iters}, "trunc": trunc}
    finally:
        ctx.close()


def run_pack(specs, stream=None):
    """Run jobs with equal pack keys as one: one context, each job's mTPQ
    sequence and probes in turn (its probes are built before the next job's
    sequence overwrites the shells), ONE blocked shifted solve over all their
    right-hand sides, and each job's spectra reweighted with its own mTPQ
    statistics (ftk_spectrum_ex). Returns one result dict per job."""
    import torch

    from . import FTK_ENOCONV, Context
    from ftk_inputs import named, omega_grid

    sp0 = specs[0]
    cl = sp0.cluster if sp0.cluster is not None else named(sp0.n_sites)
    omega = omega_grid(*sp0.omega)
    n_rhs = sum(sp.n_rhs for sp in specs)
    block = 1
    while block < n_rhs:
        block <<= 1
    stream = stream if stream is not None else torch.cuda.Stream()
    ctx = Context(cl, sp0.K, sp0.J, sp0.precision, max_rhs=block, n_saved=max(sp.n_shells for sp in specs),
                  stream=stream)
    try:
        slots, stats = [], []
        for ji, sp in enumerate(specs):
            ell = ell_for(cl, sp.K, sp.J, sp.ell)
            ctx.tpq_init(sp.seed, sp.sample, ell)
            u, lq, _ = ctx.tpq_step(sp.n_steps, sp.save_every)
            steps, _ = ctx.shells()
            stats.append((u, lq, ell, len(steps)))
            for p, (g, qi) in enumerate(sp.probes):
                for sh in range(len(steps)):
                    ctx.apply_op(sh, g, cl.momenta[qi], len(slots))
                    slots.append((ji, p, sh))
        G, it, st = ctx.shifted_cocg(list(range(len(slots))), omega, sp0.eta, tol=sp0.tol, max_iter=sp0.max_iter,
                                     allow_noconv=True)
        out = []
        for ji, sp in enumerate(specs):
            u, lq, ell, n_sh = stats[ji]
            Gj = {p: np.zeros((n_sh, len(omega)), dtype=np.complex128) for p in range(len(sp.probes))}
            itj = {p: np.zeros(n_sh, dtype=np.int64) for p in range(len(sp.probes))}
            noconv = False
            for k, (jj, p, sh) in enumerate(slots):
                if jj == ji:
                    Gj[p][sh] = G[k]
                    itj[p][sh] = it[k]
                    noconv |= st == FTK_ENOCONV and it[k] >= sp.max_iter
            spectra, trunc = {}, {}
            temps = np.asarray(sp.temps, dtype=np.float64)
            for p, probe in enumerate(sp.probes):
                S, tr = ctx.spectrum_ex(Gj[p], temps, u, lq, sp.save_every, ell)
                spectra[tuple(probe)] = S
                trunc[tuple(probe)] = tr
            out.append({"status": "noconv" if noconv else "ok", "spectra": spectra,
                        "G": {tuple(sp.probes[p]): Gj[p] for p in Gj},
                        "iters": {tuple(sp.probes[p]): itj[p] for p in itj}, "trunc": trunc, "packed": len(specs)})
        return out
    finally:
        ctx.close()


class Server:
    """Admission by footprint, up to max_slots concurrent jobs.

    runner(spec) -> dict (default: run_job on a new stream); footprint(spec)
    -> bytes (default: spec.footprint()); mem_budget: bytes (default: 90% of
    the free device memory when the server starts). pack_rhs > 0: a job being
    admitted takes waiting jobs with the same pack key along (in arrival
    order, up to pack_rhs right-hand sides in all and while their summed
    footprints fit), and the group runs as one blocked solve through
    pack_runner(specs) -> [dict] (default: run_pack).
    """

    def __init__(self, max_slots=4, mem_budget=None, runner=None, footprint=None, max_skips=8,
                 clock=time.perf_counter, pack_rhs=0, pack_runner=None):
        self.max_slots = max_slots
        self.runner = runner or run_job
        self.pack_rhs = int(pack_rhs)
        self.pack_runner = pack_runner or run_pack
        self.packs = []                   # job ids run together
        self.footprint = footprint or (lambda s: s.footprint())
        self.max_skips = max_skips
        self.clock = clock
        if mem_budget is None:
            import torch
            free, _ = torch.cuda.mem_get_info()
            mem_budget = int(0.9 * free)
        self.mem_budget = int(mem_budget)
        self._lock = threading.Condition()
        self._pending = deque()           # (job_id, spec, arrival, skips)
        self._results = {}
        self._running = {}
        self._mem_used = 0
        self._next_id = 0
        self._closed = False
        self.peak_running = 0
        self.peak_mem = 0
        self.admission_log = []           # (time, job_id, bytes in use after admission)
        self._sched = threading.Thread(target=self._loop, daemon=True)
        self._sched.start()

    # ----------------------------------------------------------- public API
    def submit(self, spec: JobSpec) -> int:
        need = self.footprint(spec)
        with self._lock:
            if self._closed:
                raise RuntimeError("server closed")
            jid = self._next_id
            self._next_id += 1
            if need > self.mem_budget:
                now = self.clock()
                self._results[jid] = JobResult(jid, f"error: footprint {need} B exceeds the budget "
                                                    f"{self.mem_budget} B", arrival=now, start=now, finish=now)
            else:
                self._pending.append([jid, spec, self.clock(), 0])
            self._lock.notify_all()
            return jid

    def result(self, job_id, timeout=None) -> JobResult:
        end = None if timeout is None else self.clock() + timeout
        with self._lock:
            while job_id not in self._results:
                left = None if end is None else end - self.clock()
                if left is not None and left <= 0:
                    raise TimeoutError(f"job {job_id} not finished")
                self._lock.wait(left)
            return self._results[job_id]

    def drain(self, timeout=None):
        with self._lock:
            ids = list(range(self._next_id))
        return [self.result(j, timeout) for j in ids]

    def stats(self):
        with self._lock:
            done = [r for r in self._results.values() if r.status in ("ok", "noconv")]
            lat = np.array([r.latency for r in done]) if done else np.zeros(0)
            spectra = sum(len(r.spectra) for r in done)
            t0 = min((r.arrival for r in done), default=0.0)
            t1 = max((r.finish for r in done), default=0.0)
            return {"jobs": len(done), "failed": len(self._results) - len(done), "spectra": spectra,
                    "spectra_per_s": spectra / (t1 - t0) if t1 > t0 else 0.0,
                    "latency_p50_s": float(np.percentile(lat, 50)) if lat.size else None,
                    "latency_p99_s": float(np.percentile(lat, 99)) if lat.size else None,
                    "peak_running": self.peak_running, "peak_mem_bytes": self.peak_mem,
                    "mem_budget_bytes": self.mem_budget}

    def close(self):
        with self._lock:
            self._closed = True
            self._lock.notify_all()
        self._sched.join()
        for t in list(self._running.values()):
            t.join()

    # ------------------------------------------------------------ scheduler
    def _pick(self):
        """Index of the next pending job to admit, or None. FIFO; a job whose
        footprint does not fit is skipped (its skip count grows) unless it
        has been passed over max_skips times, then admission waits for it."""
        free = self.mem_budget - self._mem_used
        for i, item in enumerate(self._pending):
            if self.footprint(item[1]) <= free:
                return i
            item[3] += 1
            if item[3] > self.max_skips:
                return None
        return None

    def _loop(self):
        with self._lock:
            while True:
                while not self._closed and (len(self._running) >= self.max_slots or not self._pending or
                                            self._pick_peek() is None):
                    self._lock.wait(0.05)
                if self._closed and not self._pending:
                    return
                if self._closed and len(self._running) >= self.max_slots:
                    self._lock.wait(0.05)
                    continue
                i = self._pick()
                if i is None:
                    self._lock.wait(0.05)
                    continue
                jid, spec, arrival, _ = self._pending[i]
                del self._pending[i]
                need = self.footprint(spec)
                group = [(jid, spec, arrival)]
                if self.pack_rhs > 0:
                    # compatible waiting jobs join while the right-hand sides and memory allow
                    rhs = spec.n_rhs
                    free = self.mem_budget - self._mem_used - need
                    key = spec.pack_key()
                    k = 0
                    while k < len(self._pending):
                        j2, s2, a2, _ = self._pending[k]
                        f2 = self.footprint(s2)
                        if s2.pack_key() == key and rhs + s2.n_rhs <= self.pack_rhs and f2 <= free:
                            group.append((j2, s2, a2))
                            rhs += s2.n_rhs
                            free -= f2
                            need += f2
                            del self._pending[k]
                        else:
                            k += 1
                self._mem_used += need
                self.peak_mem = max(self.peak_mem, self._mem_used)
                if len(group) == 1:
                    th = threading.Thread(target=self._work, args=(jid, spec, arrival, need), daemon=True)
                else:
                    self.packs.append([g[0] for g in group])
                    th = threading.Thread(target=self._work_pack, args=(group, need), daemon=True)
                self._running[jid] = th
                self.peak_running = max(self.peak_running, len(self._running))
                self.admission_log.append((self.clock(), jid, self._mem_used))
                th.start()

    def _pick_peek(self):
        free = self.mem_budget - self._mem_used
        for item in self._pending:
            if self.footprint(item[1]) <= free:
                return item
            if item[3] >= self.max_skips:
                return None
        return None

    def _work_pack(self, group, need):
        start = self.clock()
        try:
            outs = self.pack_runner([g[1] for g in group])
            res = [JobResult(j, o.get("status", "ok"), o.get("spectra", {}), o.get("G", {}), o.get("iters", {}),
                             o.get("trunc", {})) for (j, _, _), o in zip(group, outs)]
        except Exception as e:  # noqa: BLE001 - a failing pack must not stop the server
            res = [JobResult(j, f"error: {type(e).__name__}: {e}") for j, _, _ in group]
        fin = self.clock()
        for r, (_, _, arrival) in zip(res, group):
            r.arrival, r.start, r.finish = arrival, start, fin
        with self._lock:
            for r in res:
                self._results[r.job_id] = r
            self._mem_used -= need
            del self._running[group[0][0]]
            self._lock.notify_all()

    def _work(self, jid, spec, arrival, need):
        start = self.clock()
        try:
            out = self.runner(spec)
            res = JobResult(jid, out.get("status", "ok"), out.get("spectra", {}), out.get("G", {}),
                            out.get("iters", {}), out.get("trunc", {}))
        except Exception as e:  # noqa: BLE001 - a failing job must not stop the server
            res = JobResult(jid, f"error: {type(e).__name__}: {e}")
        res.arrival, res.start, res.finish = arrival, start, self.clock()
        with self._lock:
            self._results[jid] = res
            self._mem_used -= need
            del self._running[jid]
            self._lock.notify_all()


# ------------------------------------------------------------------ stream
def poisson_stream(n_jobs, seed=1234, rate=2.0, sizes=(12, 16, 18, 20), precisions=("fp64", "df"), n_steps=21,
                   temps=(0.005, 2.0), omega_counts=(256, 512, 1024), etas=(0.01, 0.02), max_probes=2):
    """Seeded synthetic job stream of the serving workload, scaled to one GPU
    and minutes: Poisson arrivals at `rate` jobs/s; per job a cluster size from
    `sizes`, K = -1, J ~ U[-0.3, 0.3], one or two probes (random spin component
    and momentum; at most max_probes), eta from etas, 16-64 temperatures in [temps[0],
    temps[1]], shifts on [-3, 3] (a count from omega_counts), a precision from
    `precisions`, n_steps mTPQ steps with shells every 20. Returns a list of
    (arrival offset in s, JobSpec)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for i in range(n_jobs):
        t += rng.exponential(1.0 / rate)
        n = int(rng.choice(sizes))
        n_mom = n // 2
        probes = [(int(rng.integers(0, 3)), int(rng.integers(0, n_mom)))
                  for _ in range(int(rng.integers(1, max_probes + 1)))]
        n_t = int(rng.integers(16, 65))
        spec = JobSpec(n_sites=n, K=-1.0, J=float(rng.uniform(-0.3, 0.3)), seed=int(rng.integers(1, 2**31)),
                       n_steps=n_steps, save_every=20, probes=probes,
                       omega=(-3.0, 3.0, int(rng.choice(list(omega_counts)))),
                       eta=float(rng.choice(list(etas))),
                       temps=list(np.geomspace(temps[0], temps[1], n_t)), precision=str(rng.choice(precisions)),
                       tol=1e-4, max_iter=12000, block=4)
        out.append((t, spec))
    return out


def main(argv=None):
    """Replays poisson_stream through a Server on cuda:0 and prints its stats
    (p50/p99 latency, spectra/s, peak concurrency and memory) as one JSON line."""
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=40)
    ap.add_argument("--seed", type=int, default=1234)
    ap.add_argument("--rate", type=float, default=2.0, help="arrivals per second")
    ap.add_argument("--slots", type=int, default=4)
    args = ap.parse_args(argv)
    from . import build
    build.build()
    stream = poisson_stream(args.jobs, args.seed, args.rate)
    srv = Server(max_slots=args.slots)
    t0 = time.perf_counter()
    for off, spec in stream:
        wait = t0 + off - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        srv.submit(spec)
    res = srv.drain(timeout=3600)
    srv.close()
    st = srv.stats()
    st.update({"jobs_submitted": args.jobs, "rate_per_s": args.rate, "slots": args.slots, "seed": args.seed,
               "statuses": sorted({r.status for r in res}),
               "wall_s": round(time.perf_counter() - t0, 3)})
    print(json.dumps(st), flush=True)


if __name__ == "__main__":
    main()
