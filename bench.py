"""Benchmark of the FTKomega hot path on one GB300 (or N replicas).

Workload (the 24-site plain FP64 FTKomega configuration): periodic honeycomb
3x4 cells (N = 24, dim 2^24), K = -1, J = 0.05, complex FP64 vectors. One
step = one pass of the whole hot path over one batch:
  * 21 mTPQ steps (l = 0.5) from a seeded Philox state, shells at k = 0, 20
  * S^z and S^x at momentum Q1 on both shells (4 probes)
  * one blocked shifted-COCG solve of the 4 probes, 1024 shifts on [-3, 3],
    eta = 0.01, to the paper's residual 1e-4
  * the two spectra (S^z, S^x at Q1) reweighted over the shells to 32
    temperatures in [0.005, 2]
value = algorithmic H.v bytes of the step (2 * 2^N * 16 B per vector product)
/ step time, in GB/s ("H.v GB/s"). Spectra/s, per-step latency p50/p99 and
the roofline of the dominant kernel are reported beside it.

--impl reference runs the oracle (plain C/OpenMP FP64, test infrastructure)
on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from ftk_inputs import named, omega_grid, log_temperatures  # noqa: E402

N_SITES = 24
K_COUPLING, J_COUPLING, ELL = -1.0, 0.05, 0.5
TPQ_STEPS, SAVE_EVERY = 21, 20
N_OMEGA, W_MIN, W_MAX, ETA = 1024, -3.0, 3.0, 0.01
N_T = 32
TOL, MAX_ITER = 1e-4, 10000
METRIC = "H·v GB/s vs HBM peak at N=24; spectra/s at 1e-5 err vs plain FP64; p50/p99"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class Clocks:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""

    def __init__(self):
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0],
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:6]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    import paper_1802_02854_gb300 as ftk
    from paper_1802_02854_gb300 import build as gbuild

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    gbuild.build()
    cl = named(N_SITES)
    omega = omega_grid(W_MIN, W_MAX, N_OMEGA)
    temps = log_temperatures(0.005, 2.0, N_T)
    probes = [(0, 2, 1), (1, 2, 1), (0, 0, 1), (1, 0, 1)]   # (shell, gamma, momentum index)
    kinds = [(2, 1), (0, 1)]                                 # spectra: (gamma, momentum index)
    n_rhs = len(probes)
    prec = ftk.FTK_FP64
    ctx = ftk.Context(cl, K_COUPLING, J_COUPLING, "fp64", max_rhs=n_rhs, n_saved=2)
    stream = ctx.stream
    dim = cl.dim
    hv_bytes_vec = 2 * dim * 16

    def one_step(seed):
        ctx.tpq_init(seed, rank, ELL)
        ctx.tpq_step(TPQ_STEPS, SAVE_EVERY)
        for slot, (sh, g, qi) in enumerate(probes):
            ctx.apply_op(sh, g, cl.momenta[qi], slot)
        G, it, st = ctx.shifted_cocg(list(range(n_rhs)), omega, ETA, tol=TOL, max_iter=MAX_ITER,
                                     allow_noconv=True)
        S = [ctx.spectrum(np.stack([G[2 * p], G[2 * p + 1]]), temps)[0] for p in range(len(kinds))]
        return int(np.max(it)), G, S

    for w in range(args.warmup):
        one_step(100 + w)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    times, iters_tot = [], 0
    l0 = ctx.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks() as clk:
        torch.cuda.synchronize()
        for s in range(args.steps):
            ev[s][0].record(stream)
            it, _, _ = one_step(1000 + s)
            ev[s][1].record(stream)
            iters_tot += it
        torch.cuda.synchronize()
    launches = ctx.launch_count() - l0
    for a, b in ev:
        times.append(a.elapsed_time(b) / 1e3)
    t_total = sum(times)
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([t_total], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_total = float(tt.item())
    # algorithmic H.v bytes per step: TPQ steps + blocked COCG iterations
    hv_bytes = args.steps * TPQ_STEPS * hv_bytes_vec + iters_tot * n_rhs * hv_bytes_vec
    value = world * hv_bytes / t_total / 1e9
    spectra_per_s = world * args.steps * len(kinds) / t_total

    # dominant kernel: the blocked H.V of the COCG solve (same plan, same B),
    # timed alone with CUDA events on the context stream
    v = torch.randn(n_rhs, dim, dtype=torch.complex128, device="cuda")
    out = torch.empty_like(v)
    torch.cuda.synchronize()
    for _ in range(3):
        ftk.ftk_hv(ctx.handle, v.data_ptr(), out.data_ptr(), n_rhs)
    stream.synchronize()
    reps = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ftk.ftk_hv(ctx.handle, v.data_ptr(), out.data_ptr(), n_rhs)
    e1.record(stream)
    e1.synchronize()
    t_hv = e0.elapsed_time(e1) / 1e3 / reps
    n_pass, tile_bits = ctx.plan_info()
    peak, peak_kind = peaks()
    achieved = n_rhs * hv_bytes_vec / t_hv / 1e9
    del v, out

    # end to end through the public API with host buffers
    e2e = run_e2e(ctx, cl, omega, temps, probes, kinds, args)

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * t_total / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "honeycomb24 plain FTKw FP64: 3x4 torus, K=-1, J=0.05, dim 2^24; 21 mTPQ steps "
                               "(shells k=0,20); S^z and S^x at Q1 on both shells = 4 RHS in one blocked "
                               "COCG; 1024 shifts on [-3,3], eta=0.01, tol 1e-4; 2 spectra x 32 T in [0.005,2]",
                   "n_sites": N_SITES, "n_rhs": n_rhs, "n_omega": N_OMEGA, "n_T": N_T,
                   "l2": "inputs larger than L2 (256 MiB per vector)", "parallelism": f"replicas{world}"},
        "spectra_per_s": round(spectra_per_s, 4),
        "latency_s": {"p50": round(float(np.percentile(times, 50)), 4),
                      "p99": round(float(np.percentile(times, 99)), 4)},
        "krylov_iters_per_step": iters_tot / args.steps,
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None,
                     "kernel": f"hv_pass fp64 B={n_rhs} ({n_pass} passes, tile 2^{tile_bits})",
                     "peak_kind": peak_kind, "hv_us": round(t_hv * 1e6, 2)},
        "clocks": clk.summary(),
        "e2e": e2e,
        "gpu_launches": int(launches),
    }
    if rank == 0:
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_e2e(ctx, cl, omega, temps, probes, kinds, args):
    """Same step through the public API, host state in and host spectra out."""
    import torch
    from ftk_inputs import random_state

    n_rhs = len(probes)
    psi = random_state(N_SITES, 7)             # host input (pinned copy below)
    pinned = torch.from_numpy(psi.view(np.float64)).pin_memory()
    host = pinned.numpy().view(np.complex128)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hv_iters = 0
    for s in range(max(1, min(args.steps, 2))):
        ctx.set_state(host, ELL)
        ctx.tpq_step(TPQ_STEPS, SAVE_EVERY)
        for slot, (sh, g, qi) in enumerate(probes):
            ctx.apply_op(sh, g, cl.momenta[qi], slot)
        G, it, st = ctx.shifted_cocg(list(range(n_rhs)), omega, ETA, tol=TOL, max_iter=MAX_ITER,
                                     allow_noconv=True)
        for p in range(len(kinds)):
            ctx.spectrum(np.stack([G[2 * p], G[2 * p + 1]]), temps)
        hv_iters += TPQ_STEPS + int(np.max(it)) * n_rhs
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    n = max(1, min(args.steps, 2))
    val = hv_iters * 2 * cl.dim * 16 / dt / 1e9
    return {"value": round(val, 3), "unit": "GB/s", "h2d_bytes_per_step": int(cl.dim * 16),
            "d2h_bytes_per_step": int(n_rhs * N_OMEGA * 16 + len(kinds) * N_T * N_OMEGA * 8), "steps": n}


# ------------------------------------------------------------ oracle arm
def cpu_baseline(seconds=15.0):
    """The oracle's matrix-free H.v (plain C, OpenMP, FP64) on the host cores,
    timed on a bounded sample of the workload's vector products."""
    from oracle import sparse
    from ftk_inputs import random_state

    cl = named(N_SITES)
    v = random_state(N_SITES, 3)
    sparse.hv(cl, K_COUPLING, J_COUPLING, v)
    n, t0 = 0, time.perf_counter()
    while True:
        sparse.hv(cl, K_COUPLING, J_COUPLING, v)
        n += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": round(n * 2 * cl.dim * 16 / dt / 1e9, 4), "unit": "GB/s", "cores": cores,
            "kind": "oracle", "sample": f"{n} oracle H.v products at N=24 FP64 ({dt:.1f} s)"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    per = max(3.0, args.cpu_seconds / max(1, args.steps))
    vals = []
    for _ in range(args.warmup and 1):
        cpu_baseline(1.0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(per))
    dt = time.perf_counter() - t0
    v = float(np.mean([x["value"] for x in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "honeycomb24 plain FTKw FP64 (oracle H.v on host cores)",
                       "n_sites": N_SITES},
            "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_hv_only(args):
    """A few blocked H.V launches of the bench workload (for ncu captures)."""
    import torch
    import paper_1802_02854_gb300 as ftk
    from paper_1802_02854_gb300 import build as gbuild

    gbuild.build()
    cl = named(args.hv_sites)
    prec = args.hv_prec
    ctx = ftk.Context(cl, K_COUPLING, J_COUPLING, prec, max_rhs=args.hv_rhs)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    v = torch.randn(args.hv_rhs, cl.dim, dtype=dt, device="cuda")
    out = torch.empty_like(v)
    torch.cuda.synchronize()
    for _ in range(args.hv_reps):
        ftk.ftk_hv(ctx.handle, v.data_ptr(), out.data_ptr(), args.hv_rhs)
    ctx.stream.synchronize()
    print(json.dumps({"hv_only": True, "n_sites": args.hv_sites, "prec": prec, "rhs": args.hv_rhs,
                      "plan": ctx.plan_info(), "launches": ctx.launch_count()}))
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--hv-only", action="store_true", help="only a few H.V launches (profiling)")
    ap.add_argument("--hv-sites", type=int, default=N_SITES)
    ap.add_argument("--hv-prec", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--hv-rhs", type=int, default=4)
    ap.add_argument("--hv-reps", type=int, default=4)
    args = ap.parse_args()
    if args.hv_only:
        run_hv_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
