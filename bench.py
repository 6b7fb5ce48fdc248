"""Benchmark of the FTKomega hot path on one GB300 (or N replicas).

Workload (the 24-site FTKomega configuration at scale): periodic honeycomb
3x4 cells (N = 24, dim 2^24), K = -1, J = 0.05, sites relabelled by
ftk_suggest_order. One step = one pass of the whole hot path over one batch:
  * the step's seeded initial state copied in from pinned host memory
  * 61 mTPQ steps (l = 0.5, FP64), shells k = 0, 20, 40, 60
  * S^z at momentum Q1 on the four shells (4 probes)
  * one blocked shifted-COCG solve of the 4 probes in the double-float mode
    (H.V and Krylov vectors as float hi + lo pairs on the FP32 pipe, ~48
    bits), 1024 shifts on [-3, 3], eta = 0.01, to the residual 2e-5 at which
    the spectrum is within 1e-5 of a converged FP64 solve (at the paper's
    1e-4 it is not); block plan chosen by ftk_autotune (--solve-prec picks
    another mode)
  * the spectrum reweighted over the four shells to 32 temperatures in
    [0.35, 2], the range in which the 61-step series of Eq. B1 is complete
    (its truncation flags are counted; a flagged temperature is not counted
    as a spectrum)
value = algorithmic H.v bytes of the steps (2 * 2^N * s per vector product,
s = 16 B for the FP64 mTPQ and the double-float COCG products, 8 B for FP32
ones) / device time of the steps (CUDA events on the context stream, from the
loaded state to the spectrum), in GB/s ("H.v GB/s"). e2e: the same bytes over
the host time of the same steps, the host-to-device copy of the state and the
device-to-host read of G and S included. Beside it: spectra/s, the plain FP64
single-vector FTKomega on the same GPU (same input), both spectra's error
against a converged FP64 reference (tol 1e-9), per-step latency p50/p99, a
serving stream's p50/p99, the roofline of the dominant kernel (the
double-float H.V of the solve, timed alone, against the HBM copy rate, with
its FP32-pipe fraction beside it), the FP32 H.V at 24, 26, 28 and 30 sites
and the FP64 H.V.

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

from ftk_inputs import named, omega_grid, log_temperatures, relabel, random_state  # noqa: E402

N_SITES = 24
K_COUPLING, J_COUPLING, ELL = -1.0, 0.05, 0.5
TPQ_STEPS, SAVE_EVERY = 61, 20
N_SHELLS = 4
N_OMEGA, W_MIN, W_MAX, ETA = 1024, -3.0, 3.0, 0.01
N_T, T_MIN, T_MAX = 32, 0.35, 2.0
# Krylov tolerance of the timed solve and of the plain FP64 comparison. At
# the paper's residual 1e-4 both spectra sit 2.6e-5 from the converged FP64
# reference on this workload (Krylov truncation, not arithmetic; measured), so
# the 1e-5 accuracy of the metric needs a tighter residual.
TOL, MAX_ITER = 2e-5, 14000
REF_TOL = 1e-9                  # converged FP64 reference of the error figure
METRIC = "H·v GB/s vs HBM peak at N=24; spectra/s at 1e-5 err vs plain FP64; p50/p99"
SOLVE_BYTES = {"fp64": 16, "df": 16, "mixed": 8, "fp32": 8}   # bytes per amplitude of a COCG H.v
DTYPE = {"fp64": "f64", "df": "f32x2 (double-float) H.v and Krylov vectors, f64 scalars",
         "mixed": "f32 H.v, f32x2 Krylov vectors, f64 scalars", "fp32": "f32 H.v, f64 scalars"}
# FP32-pipe operations of the double-float H.v per amplitude and term (a bond
# or the diagonal): two real double-float multiply-accumulates of 12
# operations each (FMA two-product with the cross terms: 4; two-sum and the
# lo update: 8)
DF_OPS_PER_TERM = 24
FP32_LANES_PER_SM = 128
FP64_PEAK_TFLOPS = 1.25
# DRAM bytes (read + write) of one double-float H.v of one column: ncu
# dram__bytes_read.sum + dram__bytes_write.sum summed over the three passes of
# the 24-site plan with 2^12-amplitude tiles (one column, --hv-only); valid
# for that plan of the current kernel only
DF_HV_DRAM_BYTES = 1999.0e6     # 1342.6 MB read + 656.4 MB written
DF_HV_DRAM_PLAN = (24, 3, 12)    # (sites, passes, tile bits) the counters were taken on


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


def bench_config(prec, world):
    """The workload of one step (both arms report it)."""
    return {"workload": f"honeycomb24 FTKw, {prec} solve: 3x4 torus, K=-1, J=0.05, dim 2^24; state from pinned "
                        f"host memory; {TPQ_STEPS} FP64 mTPQ steps (shells k=0,20,40,60); S^z at Q1 on the 4 shells "
                        f"= 4 RHS in one blocked COCG ({DTYPE[prec]}); 1024 shifts on [-3,3], eta=0.01, tol {TOL}; "
                        f"1 spectrum x {N_T} T in [{T_MIN},{T_MAX}]",
            "n_sites": N_SITES, "n_rhs": len(PROBES), "n_omega": N_OMEGA, "n_T": N_T, "solve_precision": prec,
            "site_order": "ftk_suggest_order", "l2": "inputs larger than L2 (128-256 MiB per vector)",
            "parallelism": f"replicas{world}"}


def job_totals(t_local, units_local, world, device):
    """Whole-job timing over the ranks: the maximum of their timed seconds and
    the sum of each of their unit counts (one collective each; world 1: the
    local values)."""
    if world == 1:
        return float(t_local), [float(u) for u in units_local]
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    uu = torch.tensor([float(u) for u in units_local], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.all_reduce(uu, op=dist.ReduceOp.SUM)
    return float(tt.item()), uu.tolist()


# ---------------------------------------------------------------- GPU arm
def bench_cluster(n=N_SITES):
    """The workload's cluster with the site labels that minimise H.v passes
    (16-byte amplitudes, one vector per launch: at N = 24 three passes for the
    double-float and FP64 products, and three for FP32 as well)."""
    import paper_1802_02854_gb300 as ftk
    cl = named(n)
    perm, _ = ftk.ftk_suggest_order(n, cl.bonds, ftk.FTK_DF, 1)
    return relabel(cl, perm)


PROBES = [(s, 2, 1) for s in range(N_SHELLS)]   # (shell, gamma, momentum index)


def run_step(ctx, cl, omega, temps, state, single=False, tol=TOL, ev=None):
    """State -> mTPQ -> probes -> blocked shifted COCG -> reweighted spectrum.
    state: complex128 host array (pinned memory for the timed steps). ev:
    (start, end) CUDA events recorded on the context stream after the state
    is loaded and after the spectrum. Returns (iters, G, S, trunc)."""
    ctx.set_state(state, ELL)
    if ev is not None:
        ev[0].record(ctx.stream)
    ctx.tpq_step(TPQ_STEPS, SAVE_EVERY)
    G = np.zeros((len(PROBES), N_OMEGA), dtype=np.complex128)
    iters = np.zeros(len(PROBES), dtype=np.int64)
    groups = [list(range(len(PROBES)))] if not single else [[p] for p in range(len(PROBES))]
    for grp in groups:
        for slot, p in enumerate(grp):
            sh, g, qi = PROBES[p]
            ctx.apply_op(sh, g, cl.momenta[qi], slot)
        Gg, it, st = ctx.shifted_cocg(list(range(len(grp))), omega, ETA, tol=tol, max_iter=MAX_ITER,
                                      allow_noconv=True)
        G[grp] = Gg
        iters[grp] = it
    S, trunc = ctx.spectrum(G, temps)
    if ev is not None:
        ev[1].record(ctx.stream)
    return iters, G, S, trunc


def products(iters, prec):
    """H.v products of one blocked solve: in the double-float mode a finished
    column stops its products; the other modes run every column of the block
    until the last one finishes."""
    it = np.asarray(iters)
    return int(it.sum()) if prec == "df" else int(it.max()) * it.size


def time_hv(ctx, torch, n_rhs, dt, reps=10, rows=None):
    """Average time of one H.V (all passes) of n_rhs vectors, CUDA events on
    the context stream; inputs larger than L2. rows: vector rows of the
    buffer (2 n_rhs for double-float: hi block, lo block)."""
    import paper_1802_02854_gb300 as ftk
    v = torch.randn(rows or n_rhs, ctx.dim, dtype=dt, device="cuda")
    out = torch.empty_like(v)
    torch.cuda.synchronize()
    for _ in range(3):
        ftk.ftk_hv(ctx.handle, v.data_ptr(), out.data_ptr(), n_rhs)
    ctx.stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(reps):
        ftk.ftk_hv(ctx.handle, v.data_ptr(), out.data_ptr(), n_rhs)
    e1.record(ctx.stream)
    e1.synchronize()
    del v, out
    return e0.elapsed_time(e1) / 1e3 / reps


def pinned_state(torch, seed):
    """The step's initial state (seeded complex Gaussian, normalised) in
    pinned host memory, as a complex128 numpy view."""
    psi = random_state(N_SITES, seed)
    pinned = torch.from_numpy(psi.view(np.float64)).pin_memory()
    return pinned, pinned.numpy().view(np.complex128)


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_serving(torch, seconds=60.0):
    """A seeded Poisson stream of spectrum jobs at N in {18, 24} through the
    continuous-batching server (own context and stream per job, admission by
    footprint): p50/p99 latency and spectra/s as the server measures them."""
    from paper_1802_02854_gb300 import serve
    jobs = serve.poisson_stream(8, seed=1234, rate=0.5, sizes=(18, 18, 18, 24), precisions=("df", "fp64"),
                                n_steps=61, temps=(T_MIN, T_MAX), omega_counts=(256,), etas=(0.02,), max_probes=1)
    srv = serve.Server(max_slots=4)
    t0 = time.perf_counter()
    for off, spec in jobs:
        wait = t0 + off - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        srv.submit(spec)
    res = srv.drain(timeout=max(600.0, 10 * seconds))
    srv.close()
    st = srv.stats()
    st.update({"jobs_submitted": len(jobs), "rate_per_s": 0.5, "slots": 4, "sizes": [18, 24], "eta": 0.02,
               "n_omega": 256, "n_steps": 61,
               "statuses": sorted({r.status for r in res}), "wall_s": round(time.perf_counter() - t0, 3)})
    return {k: (round(v, 4) if isinstance(v, float) else v) for k, v in st.items()}


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
    cl = bench_cluster()
    omega = omega_grid(W_MIN, W_MAX, N_OMEGA)
    temps = log_temperatures(T_MIN, T_MAX, N_T)
    n_rhs = len(PROBES)
    dim = cl.dim
    prec = args.solve_prec
    ctx = ftk.Context(cl, K_COUPLING, J_COUPLING, prec, max_rhs=n_rhs, n_saved=N_SHELLS)
    tuned = {"cocg": ctx.autotune(n_rhs, 0), "tpq": ctx.autotune(1, 1)}   # (tile bits, cols, us)
    stream = ctx.stream
    es = SOLVE_BYTES[prec]
    # inputs: two seeded states in pinned host memory (each rank its own seeds)
    seeds = [1000 + 2 * rank, 1001 + 2 * rank]
    host = [pinned_state(torch, sd) for sd in seeds]

    for w in range(args.warmup):
        run_step(ctx, cl, omega, temps, host[w % 2][1])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    l0 = ctx.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    S_fast, trunc_fast = None, None
    step_iters, host_times = [], []
    prods_tot = 0
    trunc_count = np.zeros(N_T, dtype=np.int64)
    with Clocks() as clk:
        torch.cuda.synchronize()
        for s in range(args.steps):
            h0 = time.perf_counter()
            it, G, S, tr = run_step(ctx, cl, omega, temps, host[s % 2][1], ev=ev[s])
            stream.synchronize()
            host_times.append(time.perf_counter() - h0)
            prods_tot += products(it, prec)
            step_iters.append(it.tolist())
            trunc_count += np.asarray(tr, dtype=np.int64)
            if s == 0:
                S_fast, trunc_fast = S, tr
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches = ctx.launch_count() - l0
    times = [a.elapsed_time(b) / 1e3 for a, b in ev]
    # algorithmic H.v bytes of the steps: FP64 mTPQ products + COCG products
    hv_bytes = args.steps * TPQ_STEPS * 2 * dim * 16 + prods_tot * 2 * dim * es
    valid_spectra = args.steps * 1 * (1.0 - float(trunc_count.max()) / args.steps)
    t_total, (hv_all, spectra_all) = job_totals(sum(times), [hv_bytes, valid_spectra], world, "cuda")
    t_host, _ = job_totals(sum(host_times), [0.0], world, "cuda")
    value = hv_all / t_total / 1e9
    spectra_per_s = spectra_all / t_total
    clocks = clk.summary()

    # dominant kernel: the blocked H.V of the solve (autotuned plan), alone
    peak, peak_kind = peaks()
    n_pass, tile_bits = ctx.plan_info()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = clocks.get("sm_max_mhz") or 2070.0
    if prec == "df":
        t_hv = time_hv(ctx, torch, n_rhs, torch.complex64, rows=2 * n_rhs)
        alg = n_rhs * 2 * dim * 16
        ops = n_rhs * dim * (len(cl.bonds) + 1) * DF_OPS_PER_TERM
        alu_peak = FP32_LANES_PER_SM * n_sm * sm_mhz * 1e6 / 1e12
        traffic = (n_rhs * DF_HV_DRAM_BYTES if DF_HV_DRAM_BYTES and (N_SITES, n_pass, tile_bits) == DF_HV_DRAM_PLAN
                   else None)
        roof = {"bound": "hbm", "achieved": round(alg / t_hv / 1e9, 2), "peak": peak, "unit": "GB/s",
                "frac": round(alg / t_hv / 1e9 / peak, 4), "traffic": traffic, "peak_kind": peak_kind,
                "kernel": f"hv_pass_df_kernel (double-float H.v, {n_rhs} columns, one per launch; tile "
                          f"2^{tile_bits}, {n_pass} passes)",
                "bytes_per_launch_set": alg, "hv_us": round(t_hv * 1e6, 2),
                "alu": {"achieved": round(ops / t_hv / 1e12, 3), "peak": round(alu_peak, 2),
                        "unit": "T ops/s (FP32 pipe, an FMA counts once)", "frac": round(ops / t_hv / 1e12 / alu_peak, 4),
                        "peak_kind": f"derived: {n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_mhz:.0f} MHz",
                        "ops_per_launch_set": ops}}
    else:
        dt = torch.complex128 if prec == "fp64" else torch.complex64
        t_hv = time_hv(ctx, torch, n_rhs, dt)
        achieved = n_rhs * 2 * dim * es / t_hv / 1e9
        roof = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None, "peak_kind": peak_kind,
                "kernel": f"hv_pass {prec} B={n_rhs} (one H.v = all passes; tile 2^{tile_bits}, "
                          f"{tuned['cocg'][1]} columns per launch)", "hv_us": round(t_hv * 1e6, 2)}
    # the metric's H.v against the HBM peak: FP32, one vector, all passes
    ctx1 = ftk.Context(cl, K_COUPLING, J_COUPLING, "fp32", max_rhs=1)
    t_hv1 = time_hv(ctx1, torch, 1, torch.complex64)
    p1 = ctx1.plan_info()
    ctx1.close()
    # the FP64 H.v (mTPQ and the plain FP64 solve) against the FP64 pipe:
    # 2 DFMA (4 flops) per amplitude and term (bonds + diagonal)
    ctx2 = ftk.Context(cl, K_COUPLING, J_COUPLING, "fp64", max_rhs=1)
    t_hv64 = time_hv(ctx2, torch, 1, torch.complex128)
    p64 = ctx2.plan_info()
    ctx2.close()
    fl64 = dim * (len(cl.bonds) + 1) * 4
    roof["hv_fp64_b1"] = {"us": round(t_hv64 * 1e6, 2), "gbs": round(2 * dim * 16 / t_hv64 / 1e9, 2),
                          "hbm_frac": round(2 * dim * 16 / t_hv64 / 1e9 / peak, 4),
                          "tflops": round(fl64 / t_hv64 / 1e12, 3),
                          "fp64_frac": round(fl64 / t_hv64 / 1e12 / FP64_PEAK_TFLOPS, 4),
                          "fp64_peak": FP64_PEAK_TFLOPS, "fp64_peak_kind": "nominal GB300 FP64", "passes": p64[0]}
    roof["hv_fp32_b1"] = {"us": round(t_hv1 * 1e6, 2), "gbs": round(2 * dim * 8 / t_hv1 / 1e9, 2),
                          "frac": round(2 * dim * 8 / t_hv1 / 1e9 / peak, 4), "peak": peak,
                          "peak_kind": peak_kind, "passes": p1[0]}

    # the metric's H.v over the cluster sizes of the workloads (24-30 sites):
    # FP32, one vector, sites relabelled for FP32 tiles, all passes
    by_n = {}
    if not args.no_n_sweep:
        for n in (26, 28, 30):
            cn = named(n)
            perm_n, _ = ftk.ftk_suggest_order(n, cn.bonds, ftk.FTK_FP32, 1)
            cn = relabel(cn, perm_n)
            cx = ftk.Context(cn, K_COUPLING, J_COUPLING, "fp32", max_rhs=1)
            t_n = time_hv(cx, torch, 1, torch.complex64, reps=4)
            gbs_n = 2 * (1 << n) * 8 / t_n / 1e9
            by_n[str(n)] = {"us": round(t_n * 1e6, 1), "gbs": round(gbs_n, 1), "frac": round(gbs_n / peak, 4),
                            "passes": cx.plan_info()[0], "tile_bits": cx.plan_info()[1]}
            cx.close()
            torch.cuda.empty_cache()
    roof["hv_fp32_by_n"] = by_n

    # the batched configuration's knob: FP64 blocked H.V time per column
    # against the block width (tile size and column chunk autotuned per width)
    blocked = {"B": [], "us_per_column": [], "plan": []}
    if not args.no_block_sweep:
        for B in (1, 4, 8, 16, 32):
            cb = ftk.Context(cl, K_COUPLING, J_COUPLING, "fp64", max_rhs=B)
            tb_, cols_, _ = cb.autotune(B, 0)
            t_b = time_hv(cb, torch, B, torch.complex128, reps=3)
            blocked["B"].append(B)
            blocked["us_per_column"].append(round(t_b * 1e6 / B, 1))
            blocked["plan"].append([tb_, cols_, cb.plan_info()[0]])
            cb.close()
    roof["hv_fp64_blocked"] = blocked

    # plain FP64 single-vector FTKomega on the same GPU and input (timed step
    # 0's state), and a converged FP64 reference (tol 1e-9) for the errors
    ctx64 = ftk.Context(cl, K_COUPLING, J_COUPLING, "fp64", max_rhs=n_rhs, n_saved=N_SHELLS)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it64, G64, S64, _ = run_step(ctx64, cl, omega, temps, host[0][1], single=True)
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t0
    itr, Gr, S_ref, tr_ref = run_step(ctx64, cl, omega, temps, host[0][1], tol=REF_TOL)
    ctx64.close()
    err_fast, err_fp64 = rel_err(S_fast, S_ref), rel_err(S64, S_ref)

    # serving: a short Poisson stream of jobs at N = 18 and 24
    serving = None if args.no_serving else run_serving(torch)

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * t_total / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[prec], "data": "synthetic",
        "config": dict(bench_config(prec, world), autotune=tuned),
        "spectra_per_s": round(spectra_per_s, 4),
        "trunc": {"per_T": trunc_count.tolist(), "flagged_T": int((trunc_count > 0).sum()),
                  "note": "steps whose 61-step series of Eq. B1 is truncated at each T (0: every spectrum valid)"},
        "spectrum_rel_err": {"fast_vs_ref": err_fast, "plain_fp64_vs_ref": err_fp64,
                             "fast_vs_plain_fp64": rel_err(S_fast, S64), "ref": f"FP64 blocked, tol {REF_TOL}",
                             "ref_krylov_iters": itr.tolist(),
                             "norm": "||S - S_ref||_2 / ||S_ref||_2 over (omega, T), timed step 0's input"},
        "plain_fp64": {"spectra_per_s": round(1.0 / t64, 5), "seconds": round(t64, 3), "krylov_iters": it64.tolist(),
                       "speedup": round(spectra_per_s / world * t64, 3),
                       "speedup_same_input": round(t64 / times[0], 3),
                       "note": "single-vector FP64 solves of the same probes at the same tol, step 0's input"},
        "krylov_iters_by_step": step_iters,
        "latency_s": {"p50": round(float(np.percentile(times, 50)), 4),
                      "p99": round(float(np.percentile(times, 99)), 4), "what": "device time per step"},
        "serving": serving,
        "roofline": roof,
        "clocks": clocks,
        "e2e": {"value": round(hv_all / t_host / 1e9, 3), "unit": "GB/s", "h2d_bytes_per_step": int(dim * 16),
                "d2h_bytes_per_step": int(n_rhs * N_OMEGA * 16 + N_T * N_OMEGA * 8 + N_T * 4),
                "steps": args.steps, "what": "host time of the same timed steps, state H2D and G, S D2H included"},
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
            "config": bench_config(args.solve_prec, world),
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
    cl = bench_cluster(args.hv_sites)
    prec = args.hv_prec
    ctx = ftk.Context(cl, K_COUPLING, J_COUPLING, prec, max_rhs=args.hv_rhs)
    if args.hv_autotune:
        ctx.autotune(args.hv_rhs, 0)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    v = torch.randn(args.hv_rhs * (2 if prec == "df" else 1), cl.dim, dtype=dt, device="cuda")
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
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving stream")
    ap.add_argument("--no-block-sweep", action="store_true", help="skip the FP64 block-width sweep")
    ap.add_argument("--no-n-sweep", action="store_true", help="skip the FP32 H.v at 26, 28 and 30 sites")
    ap.add_argument("--hv-only", action="store_true", help="only a few H.V launches (profiling)")
    ap.add_argument("--hv-sites", type=int, default=N_SITES)
    ap.add_argument("--hv-prec", default="fp32", choices=["fp64", "fp32", "df"])
    ap.add_argument("--hv-rhs", type=int, default=4)
    ap.add_argument("--hv-reps", type=int, default=4)
    ap.add_argument("--hv-autotune", action="store_true")
    ap.add_argument("--max-iter", type=int, default=0, help="cap Krylov iterations (profiling runs)")
    ap.add_argument("--solve-prec", default="df", choices=["df", "mixed", "fp64", "fp32"],
                    help="precision mode of the blocked COCG solve")
    args = ap.parse_args()
    global MAX_ITER
    if args.max_iter > 0:
        MAX_ITER = args.max_iter
    if args.hv_only:
        run_hv_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
