"""Benchmark of the two-site DMRG hot path on GB300.

Workload (default): 1D Hubbard chain, L = 32 sites, t = 1, U = 4, open ends, half filling,
Sz = 0, bond dimension M = 500, FP64 wavefunction.  One step = one full two-site sweep
(forward and backward half) through the C-ABI (``b2_sweep``): every H_eff . psi product,
H_eff diagonal, Davidson, density-matrix eigensolve, truncation and environment update.
Inputs are synthetic (seeded integrals and random initial MPS).  Untimed setup sweeps run
from the random MPS until every bond has reached M and the sweep energy has settled (change
below 1e-8 Eh, at most 14 sweeps), so that the W warm-up and K timed sweeps are sweeps at
bond dimension M.

metric/value: algorithmic H_eff . psi FLOP/s over the whole sweep (flops of the block
GEMMs the contraction performs, summed over every product in the sweep, divided by the
sweep's device time).  e2e: the same metric when each step also imports the MPS from host
memory, builds the environments and exports the MPS back (host copies inside the timed
region).  roofline: the kernel with the larger device time in the timed sweeps -- the
H_eff contraction (algorithmic block-GEMM flops) or the truncation eigensolver (12 m_a + 6 m
flops per applied Jacobi rotation, m_a the rows active in that sweep) -- timed by CUDA
events inside the library, against the FP64 peak measured on this GPU with cuBLAS DGEMM;
roofline_other: the other one.

``--impl reference`` times the CPU oracle (``oracle/``) on a bounded sample of the same
workload (H_eff . psi products at the middle window) on the host cores.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under torchrun with one
process per GPU (independent replicas: the sweep does not shard).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H_eff·ψ TFLOP/s & sweep time, mixed-prec vs FP64 on GB300 at |ΔE|≤1e-6 Eh"
WORKLOAD = dict(name="hubbard_L32_U4_halffilling_M500_sweep", L=32, t=1.0, U=4.0, M=500,
                mps_seed=1132)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "bf16x3", "tf32x3"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the split-precision sweeps compared with FP64 on the same state")
    ap.add_argument("--no-window", action="store_true",
                    help="skip the n=36 middle-window leg (products at M=1000/2000, Davidson "
                         "at M=1000 in FP64 and in split precision)")
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work")
    ap.add_argument("--window-m", type=int, default=0,
                    help="window_M*: bond dimension of the n=36 window (default: from the name)")
    ap.add_argument("--workload", default="sweep",
                    choices=["sweep", "window_M1000", "window_M2000", "batch64", "batch64_sweeps",
                             "grad_n24", "eig_batch", "sweep_n36"],
                    help="sweep: Hubbard L=32 M=500 full sweep (default); window_M*: middle "
                         "window of the n=36 ab initio system, FP64 vs split precision; "
                         "batch64: 64 independent problems, grouped vs one-by-one launches; "
                         "grad_n24: integral gradient (1- and 2-RDM) at n=24, M=500; "
                         "eig_batch: the truncation eigensolver alone on one truncation-shaped "
                         "batch of graded density matrices; sweep_n36: full sweeps of the n=36 "
                         "ab initio system at M = --window-m (default 1000), precision --prec")
    ap.add_argument("--batch", type=int, default=64, help="problems of the batch64 workloads")
    ap.add_argument("--sweeps", type=int, default=6, help="batch64_sweeps: sweeps per problem")
    ap.add_argument("--one-by-one", action="store_true",
                    help="batch64_sweeps: also run every problem's sweeps one problem at a time")
    ap.add_argument("--davidson", action="store_true",
                    help="window_M*: also solve the window (split precision to |r|^2 <= 1e-7, "
                         "then FP64 from that vector) and report |dE|; several minutes")
    return ap.parse_args()


def aggregate_ranks(t_tot, flops, device):
    """Whole-job figures of N independent replicas: time = max over ranks, flops = sum over
    ranks (one process per GPU; identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t_tot, flops
    t = torch.tensor([t_tot], dtype=torch.float64, device=device)
    f = torch.tensor([flops], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(f, op=dist.ReduceOp.SUM)
    return float(t[0]), float(f[0])


def dist_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def workload_inputs():
    from synth import hubbard_integrals, occupancies, random_mps, sector_sizes
    w = WORKLOAD
    h, eri = hubbard_integrals(w["L"], w["t"], w["U"])
    bonds = sector_sizes(w["L"], w["L"], 0, w["M"], occupancies(w["L"], w["L"], "hubbard"))
    sites = random_mps(bonds, seed=w["mps_seed"])
    return h, eri, bonds, sites


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows)}


def measured_peaks(torch):
    """FP64 and TF32 peaks of this GPU (cuBLAS through torch.matmul, 8192^3, float64 /
    float32 with TF32 allowed, best of 5) and the measured HBM / bf16 figures."""
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks.update(json.load(f))
    except OSError:
        pass
    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = 0.0
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    peaks["fp64_tflops_measured"] = best
    del a, b
    # TF32: float32 matmul with TF32 tensor cores allowed (same protocol)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    a = torch.randn(n, n, dtype=torch.float32, device="cuda")
    b = torch.randn(n, n, dtype=torch.float32, device="cuda")
    torch.matmul(a, b)
    best = 0.0
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    torch.backends.cuda.matmul.allow_tf32 = prev
    peaks["tf32_tflops_measured"] = best
    del a, b
    torch.cuda.empty_cache()
    return peaks


def oracle_sample(budget_s):
    """The CPU oracle on a bounded sample of the workload: H_eff . psi products at the
    middle window (sites 15, 16) of the workload's random MPS centred there, and the
    algorithmic flops of one product counted by the oracle itself (block-sparse form of its
    own term list).  Returns (seconds per product, products, setup seconds, flops)."""
    import numpy as np
    from oracle import dmrg, mpo
    h, eri, bonds, sites = workload_inputs()
    from synth import random_mps
    c = WORKLOAD["L"] // 2 - 1
    sites_c = random_mps(bonds, seed=WORKLOAD["mps_seed"], center=c)
    t0 = time.perf_counter()
    d = dmrg.DMRG(mpo.MPO(h, eri), bonds, sites_c, center=c)
    H = d.heff(c)
    setup = time.perf_counter() - t0
    flops = H.algorithmic_flops(d.lab[c], d.lab[c + 2])
    x = d.psi
    times = []
    t_start = time.perf_counter()
    while True:
        t1 = time.perf_counter()
        x = H.apply(x)
        x /= np.linalg.norm(x)
        times.append(time.perf_counter() - t1)
        if time.perf_counter() - t_start > budget_s or len(times) >= 50:
            break
    return statistics.median(times), len(times), setup, flops


def gpu_middle_window_product(b2, torch, ctx):
    """The same sample on the GPU: FP64 H_eff . psi products at window (15, 16) of the
    workload's random MPS centred there (the oracle sample's input), timed with CUDA events
    on the context stream.  Returns (ms per product, library flops, oracle-definition
    flops are not computed here)."""
    from synth import random_mps
    h, eri, bonds, sites = workload_inputs()
    c = WORKLOAD["L"] // 2 - 1
    sites_c = random_mps(bonds, seed=WORKLOAD["mps_seed"], center=c)
    m = b2.b2_build_mpo(ctx, h, eri, 0.0, WORKLOAD["L"], 0)
    s = b2.b2_mps_import(ctx, bonds, sites_c, WORKLOAD["L"], 0, center=c)
    env = b2.b2_env_init(ctx, m, s, center=c)
    n_elem, _ = b2.b2_psi_layout(ctx, env, c)
    x = torch.empty(n_elem, dtype=torch.float64, device="cuda")
    b2.b2_psi_from_mps(ctx, env, c, x)
    y = torch.empty_like(x)
    fl = b2.b2_heff_apply(ctx, env, c, x, y)
    torch.cuda.synchronize()
    reps = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(reps):
        b2.b2_heff_apply(ctx, env, c, x, y)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    b2.b2_free_env(env)
    b2.b2_free_mps(s)
    b2.b2_free_mpo(m)
    return e0.elapsed_time(e1) / reps, fl


def cpu_cores():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        blas = [i.get("num_threads") for i in info if i.get("user_api") == "blas"]
        if blas:
            return int(blas[0])
    except Exception:
        pass
    return os.cpu_count()


def run_reference(args):
    """The oracle as the reference arm: each step is a bounded sample of the workload
    (H_eff . psi products at the middle window, timed on the host cores); the flops of one
    product are counted by the oracle (block-sparse form of its own term list).  Nothing of
    the GPU library is loaded."""
    rank, world, local = dist_info()
    if rank != 0:
        return
    budget = max(2.0, args.cpu_budget)
    sec, nprod, setup, fl = oracle_sample(budget)
    value = fl / sec / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "L": WORKLOAD["L"], "U": WORKLOAD["U"],
                       "M": WORKLOAD["M"], "sample": "H_eff.psi at the middle window"},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cpu_cores(),
                             "kind": "oracle",
                             "sample": "%d oracle H_eff.psi products at window %d of the "
                                       "workload's random MPS (setup %.1f s); %.4g flops per "
                                       "product (oracle count)" % (nprod, WORKLOAD["L"] // 2 - 1,
                                                                   setup, fl)},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def window_leg(b2, torch, ctx, M, davidson, reps, peaks):
    """Middle window (sites 17, 18) of the n = 36, N = 36 ab initio system (60 Cholesky
    vectors decaying as exp(-|p-q|/6), seed 2) at bond dimension M from a random MPS centred
    there.  Times single H_eff . psi products in FP64, bf16 x3 and tf32 x3 (CUDA events on
    the context stream, L2 flushed before each timing) and their relative difference to
    FP64.  With davidson: the window's ground state from a common start vector (an FP64
    Davidson to |r|^2 <= 1e-5 from the MPS's psi, untimed) to |r|^2 <= 1e-10 in FP64 and
    with split products refined in FP64, with times, products and |dE|."""
    from synth import config_integrals, occupancies, random_mps, sector_sizes
    h, eri, N, tsz, kind = config_integrals("abinitio_n36")
    n = h.shape[0]
    c = n // 2 - 1
    t0 = time.perf_counter()
    bonds = sector_sizes(n, N, tsz, M, occupancies(n, N, kind))
    sites = random_mps(bonds, seed=2 + 100, center=c)
    mpo_h = b2.b2_build_mpo(ctx, h, eri, 0.0, N, tsz)
    mps_h = b2.b2_mps_import(ctx, bonds, sites, N, tsz, center=c)
    env = b2.b2_env_init(ctx, mpo_h, mps_h, center=c)
    setup = time.perf_counter() - t0
    n_elem, n_blk = b2.b2_psi_layout(ctx, env, c)
    psi0 = torch.empty(n_elem, dtype=torch.float64, device="cuda")
    b2.b2_psi_from_mps(ctx, env, c, psi0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    res = {"config": {"n": n, "n_elec": N, "M": M, "window": [c, c + 1], "psi_elements": n_elem,
                      "psi_blocks": n_blk}, "setup_s": setup}
    bf16_peak = peaks.get("bf16_tflops", 1887.4)
    ys = {}
    for name, prec in (("fp64", b2.B2_FP64), ("bf16x3", b2.B2_BF16X3), ("tf32x3", b2.B2_TF32X3)):
        y = torch.empty_like(psi0)
        fl = b2.b2_heff_apply(ctx, env, c, psi0, y, prec=prec)   # builds / splits once
        ms = []
        if prec == b2.B2_BF16X3:   # profiler range: the timed split-precision products
            torch.cuda.synchronize()
            torch.cuda.cudart().cudaProfilerStart()
        for _ in range(1 if prec == b2.B2_FP64 else reps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(ctx.stream)
            b2.b2_heff_apply(ctx, env, c, psi0, y, prec=prec)
            e1.record(ctx.stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        if prec == b2.B2_BF16X3:
            torch.cuda.cudart().cudaProfilerStop()
        t = statistics.median(ms)
        ys[name] = y
        r = {"ms": t, "algo_flops": fl, "effective_tflops": fl / (t * 1e-3) / 1e12}
        if prec != b2.B2_FP64:
            pipe = 3 * fl / (t * 1e-3) / 1e12
            peak = bf16_peak if prec == b2.B2_BF16X3 else bf16_peak / 2   # tf32: half the rate
            r.update({"tensor_pipe_tflops": pipe, "tensor_peak_tflops": peak,
                      "tensor_frac": pipe / peak,
                      "rel_err_vs_fp64": float((y - ys["fp64"]).norm() / ys["fp64"].norm()),
                      "speedup_vs_fp64": res["fp64"]["ms"] / t})
        res[name] = r
    if davidson:
        p = psi0.clone()
        b2.b2_davidson(ctx, env, c, p, max_iter=200, max_subspace=40, conv_tol=1e-5)
        dav = {"conv_tol": 1e-10, "start": "FP64 Davidson to |r|^2 <= 1e-5 from the MPS's psi"}
        for name, prec in (("fp64", b2.B2_FP64), ("tf32x3", b2.B2_TF32X3), ("bf16x3", b2.B2_BF16X3)):
            q = p.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e, nmv, r2 = b2.b2_davidson(ctx, env, c, q, max_iter=200, max_subspace=40,
                                        conv_tol=1e-10, prec=prec, refine_max=20)
            torch.cuda.synchronize()
            dav[name] = {"seconds": time.perf_counter() - t0, "energy": e, "n_matvec": nmv,
                         "resid2": r2}
        for name in ("tf32x3", "bf16x3"):
            dav[name]["dE_vs_fp64"] = abs(dav[name]["energy"] - dav["fp64"]["energy"])
            dav[name]["speedup_vs_fp64"] = dav["fp64"]["seconds"] / dav[name]["seconds"]
        res["davidson"] = dav
    del flush
    b2.b2_free_env(env)
    b2.b2_free_mps(mps_h)
    b2.b2_free_mpo(mpo_h)
    torch.cuda.empty_cache()
    return res


def run_window(args):
    """Middle window of the n = 36 ab initio system at M = 1000 or 2000 (window_leg): the
    split-precision product is the line's value; with --davidson also the window solves."""
    import torch
    from paper_2310_03920_gb300 import b2
    M = args.window_m or (1000 if args.workload == "window_M1000" else 2000)
    ctx = b2.Context(0)
    peaks = measured_peaks(torch)
    b2.b2_profile(ctx, True)
    with ClockSampler(0) as clk:
        res = window_leg(b2, torch, ctx, M, args.davidson, max(3, args.steps), peaks)
    prof = b2.b2_profile_read(ctx)
    b2.b2_profile(ctx, False)
    best = max(("bf16x3", "tf32x3"), key=lambda k: res[k]["effective_tflops"])
    line = {"metric": METRIC, "value": res[best]["effective_tflops"], "unit": "TFLOP/s",
            "n_gpus": 1, "steps": max(3, args.steps), "warmup": 1, "ms_per_step": res[best]["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": best,
            "data": "synthetic",
            "config": dict(workload="abinitio_n36_N36_M%d_middle_window" % M,
                           l2="flushed before each product (256 MB write)", **res["config"]),
            "window": res, "gpu_launches": int(prof["launches"]), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_batch(args):
    """64 independent problems (Hubbard L in [12, 40], U in [1, 8]; ab initio n in [10, 24];
    M in [100, 800]; ``synth.batch_problem``), each from a random MPS centred at its middle
    window.  Times (a) the H_eff products of all problems one launch each and (b) one
    grouped launch over all problems (b2_heff_apply_batched), in FP64 and in split precision,
    and the Davidson solves of all middle windows one by one vs in lockstep
    (b2_davidson_batched, 12 products at most)."""
    import numpy as np
    import torch
    from paper_2310_03920_gb300 import b2
    from synth import batch_problem, occupancies, random_mps, sector_sizes
    ctx = b2.Context(0)
    t0 = time.perf_counter()
    probs = []
    for j in range(args.batch):
        pr = batch_problem(j)
        n, N, tsz = pr["n"], pr["n_elec"], pr["two_sz"]
        c = n // 2 - 1
        kind = "hubbard" if pr["kind"] == "hubbard" else "ab_initio"
        bonds = sector_sizes(n, N, tsz, pr["M"], occupancies(n, N, kind))
        sites = random_mps(bonds, seed=pr["seed"], center=c)
        mpo = b2.b2_build_mpo(ctx, pr["h"], pr["eri"], 0.0, N, tsz)
        mps = b2.b2_mps_import(ctx, bonds, sites, N, tsz, center=c)
        env = b2.b2_env_init(ctx, mpo, mps, center=c)
        n_elem, _ = b2.b2_psi_layout(ctx, env, c)
        psi = torch.empty(n_elem, dtype=torch.float64, device="cuda")
        b2.b2_psi_from_mps(ctx, env, c, psi)
        probs.append({"mpo": mpo, "mps": mps, "env": env, "site": c, "psi": psi,
                      "out": torch.empty_like(psi), "kind": pr["kind"], "n": n, "M": pr["M"]})
    t_setup = time.perf_counter() - t0
    envs = [p["env"] for p in probs]
    sites = [p["site"] for p in probs]
    psis = [p["psi"] for p in probs]
    outs = [p["out"] for p in probs]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    reps = max(3, args.steps)

    def timed(fn):
        fn()                                   # builds window programs, precombines
        ms = []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fl = fn()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.median(ms)), fl

    res = {}
    for name, prec in (("fp64", b2.B2_FP64), ("bf16x3", b2.B2_BF16X3)):
        ms_one, fl = timed(lambda: sum(b2.b2_heff_apply(ctx, p["env"], p["site"], p["psi"], p["out"],
                                                        prec=prec) for p in probs))
        b2.b2_profile(ctx, True)
        ms_grp, fl_g = timed(lambda: b2.b2_heff_apply_batched(ctx, envs, sites, psis, outs, prec=prec))
        prof = b2.b2_profile_read(ctx)
        b2.b2_profile(ctx, False)
        res[name] = {"algo_flops": fl, "one_by_one_ms": ms_one, "grouped_ms": ms_grp,
                     "one_by_one_tflops": fl / (ms_one * 1e-3) / 1e12,
                     "grouped_tflops": fl_g / (ms_grp * 1e-3) / 1e12,
                     "speedup": ms_one / ms_grp,
                     "grouped_launches_per_call": prof["launches"] / (reps + 1)}
    # Davidson of every middle window: one by one vs lockstep
    dav = {}
    for name in ("one_by_one", "lockstep"):
        ys = [p["psi"].clone() for p in probs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if name == "one_by_one":
            out = [b2.b2_davidson(ctx, p["env"], p["site"], y, max_iter=12, max_subspace=30,
                                  conv_tol=1e-10) for p, y in zip(probs, ys)]
            energies = [o[0] for o in out]
            nmv = int(sum(o[1] for o in out))
        else:
            e, n_mv, _ = b2.b2_davidson_batched(ctx, envs, sites, ys, max_iter=12, max_subspace=30,
                                                conv_tol=1e-10)
            energies, nmv = list(e), int(n_mv.sum())
        torch.cuda.synchronize()
        dav[name] = {"seconds": time.perf_counter() - t0, "n_matvec": nmv, "energies": energies}
    same = all(a == b for a, b in zip(dav["one_by_one"]["energies"], dav["lockstep"]["energies"]))
    for d in dav.values():
        d.pop("energies")
    peaks = measured_peaks(torch)
    g = res["fp64"]
    line = {"metric": METRIC, "value": g["grouped_tflops"], "unit": "TFLOP/s", "n_gpus": 1,
            "steps": reps, "warmup": 1, "ms_per_step": g["grouped_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batch%d_middle_windows" % len(probs), "problems": len(probs),
                       "hubbard": sum(p["kind"] == "hubbard" for p in probs),
                       "ab_initio": sum(p["kind"] != "hubbard" for p in probs),
                       "n_range": [min(p["n"] for p in probs), max(p["n"] for p in probs)],
                       "M_range": [min(p["M"] for p in probs), max(p["M"] for p in probs)],
                       "l2": "flushed between steps (256 MB write)"},
            "heff": res, "davidson": dav, "lockstep_energies_identical": same,
            "fp64_peak_tflops": peaks.get("fp64_tflops_measured"), "setup_s": t_setup}
    print(json.dumps(line), flush=True)
    for p in probs:
        b2.b2_free_env(p["env"])
        b2.b2_free_mps(p["mps"])
        b2.b2_free_mpo(p["mpo"])
    ctx.close()


def run_batch_sweeps(args):
    """All problems of the batch (synth.batch_problem: Hubbard L in [12, 40], U in [1, 8];
    ab initio n in [10, 24]; M in [100, 800]) run to the end of --sweeps two-site sweeps at
    their own bond dimension, from random MPS (b2_mps_random, seed of the problem) in
    lockstep (b2_sweep_batched_dims: one grouped H_eff launch per Davidson iteration over
    every problem still iterating).  value = the problems' H_eff flops / time to all done."""
    import numpy as np
    import torch
    from paper_2310_03920_gb300 import b2
    from synth import batch_problem
    ctx = b2.Context(0)
    probs = []
    t0 = time.perf_counter()
    for j in range(args.batch):
        pr = batch_problem(j)
        n, N, tsz = pr["n"], pr["n_elec"], pr["two_sz"]
        occ = np.full(n, 0.5) if pr["kind"] == "hubbard" else None
        mpo = b2.b2_build_mpo(ctx, pr["h"], pr["eri"], 0.0, N, tsz)
        probs.append({"mpo": mpo, "occ": occ, "seed": pr["seed"], "M": pr["M"], "n": n,
                      "kind": pr["kind"]})
    t_mpo = time.perf_counter() - t0

    def fresh():
        envs = []
        for p in probs:
            p["mps"] = b2.b2_mps_random(ctx, p["mpo"], p["M"], p["occ"], p["seed"])
            envs.append(b2.b2_env_init(ctx, p["mpo"], p["mps"], 0))
        return envs

    def release(envs):
        for p, e in zip(probs, envs):
            b2.b2_free_env(e)
            b2.b2_free_mps(p["mps"])

    dims = [[p["M"]] * args.sweeps for p in probs]
    envs = fresh()
    torch.cuda.synchronize()
    b2.b2_profile(ctx, True)
    t0 = time.perf_counter()
    res = b2.b2_sweep_batched_dims(ctx, envs, dims, prec=b2.PRECISIONS[args.prec])
    torch.cuda.synchronize()
    t_lock = time.perf_counter() - t0
    prof = b2.b2_profile_read(ctx)
    b2.b2_profile(ctx, False)
    flops = sum(r["matvec_flops"] for pr in res for r in pr)
    energies = [pr[-1]["energy"] for pr in res]
    release(envs)
    out = {"lockstep_s": t_lock, "lockstep_tflops": flops / t_lock / 1e12,
           "heff_device_ms": prof["heff_ms"], "eig_device_ms": prof["eig_ms"],
           "gpu_launches": int(prof["launches"])}
    if args.one_by_one:
        envs = fresh()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e1 = []
        for p, e in zip(probs, envs):
            r = b2.b2_sweep(ctx, p["mpo"], p["mps"], e, [p["M"]] * args.sweeps,
                            prec=b2.PRECISIONS[args.prec])
            e1.append(r[-1]["energy"])
        torch.cuda.synchronize()
        out["one_by_one_s"] = time.perf_counter() - t0
        out["speedup"] = out["one_by_one_s"] / t_lock
        out["energies_identical"] = all(a == b for a, b in zip(energies, e1))
        release(envs)
    line = {"metric": METRIC, "value": out["lockstep_tflops"], "unit": "TFLOP/s", "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": t_lock * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.prec == "fp64" else args.prec, "data": "synthetic",
            "config": {"workload": "batch%d_%dsweeps_lockstep" % (len(probs), args.sweeps),
                       "prec": args.prec,
                       "problems": len(probs),
                       "hubbard": sum(p["kind"] == "hubbard" for p in probs),
                       "ab_initio": sum(p["kind"] != "hubbard" for p in probs),
                       "n_range": [min(p["n"] for p in probs), max(p["n"] for p in probs)],
                       "M_range": [min(p["M"] for p in probs), max(p["M"] for p in probs)]},
            "batch": out, "mpo_build_s": t_mpo,
            "final_energies": {"min": min(energies), "max": max(energies)}}
    print(json.dumps(line), flush=True)
    for p in probs:
        b2.b2_free_mpo(p["mpo"])
    ctx.close()


def run_sweep_n36(args):
    """Full two-site sweeps (--sweeps of them) of the n = 36, N = 36 ab initio system
    (the window leg's integrals) at bond dimension M = --window-m (default 1000) from a random
    MPS centred at site 0 (sector recipe, seed 2), in precision --prec (split precision with
    FP64 refinement, or FP64).  Reports per sweep: wall time, energy, products, Davidson and
    split times, largest bond; the time includes each window's host program build."""
    import torch
    from paper_2310_03920_gb300 import b2
    from synth import config_integrals, occupancies, random_mps, sector_sizes
    h, eri, N, tsz, kind = config_integrals("abinitio_n36")
    n = h.shape[0]
    M = args.window_m or 1000
    ctx = b2.Context(0)
    t0 = time.perf_counter()
    bonds = sector_sizes(n, N, tsz, M, occupancies(n, N, kind))
    sites = random_mps(bonds, seed=2 + 100, center=0)
    mpo = b2.b2_build_mpo(ctx, h, eri, 0.0, N, tsz)
    mps = b2.b2_mps_import(ctx, bonds, sites, N, tsz, center=0)
    env = b2.b2_env_init(ctx, mpo, mps, center=0)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    prec = b2.PRECISIONS[args.prec]
    res = b2.b2_sweep(ctx, mpo, mps, env, [M] * max(1, args.sweeps), prec=prec)
    sweeps = [{"seconds": r["seconds"], "energy": r["energy"], "n_matvec": r["n_matvec"],
               "t_davidson": r["t_davidson"], "t_split": r["t_split"], "max_bond": r["max_bond"],
               "discarded_weight": r["discarded_weight"], "matvec_flops": r["matvec_flops"]}
              for r in res]
    sec = sum(r["seconds"] for r in sweeps)
    line = {"metric": METRIC, "value": sum(r["matvec_flops"] for r in sweeps) / sec / 1e12,
            "unit": "TFLOP/s", "n_gpus": 1, "steps": len(sweeps), "warmup": 0,
            "ms_per_step": sec * 1e3 / len(sweeps), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.prec == "fp64" else args.prec,
            "data": "synthetic",
            "config": {"workload": "abinitio_n36_N36_M%d_sweep" % M, "n": n, "n_elec": N, "M": M,
                       "start": "random MPS (sector recipe) centred at site 0"},
            "setup_s": setup, "sweeps": sweeps,
            "peak_device_gb": torch.cuda.max_memory_allocated() / 1e9}
    print(json.dumps(line), flush=True)
    b2.b2_free_env(env)
    b2.b2_free_mps(mps)
    b2.b2_free_mpo(mpo)
    ctx.close()


def run_grad(args):
    """Integral gradient dE/dh, dE/d(pq|rs) (spin-traced 1- and 2-RDM) of an n = 24,
    N = 24 ab initio MPS at M = 500 (random MPS from the sector recipe, seeded): times
    b2_rdm_grad end to end (gradient MPO build, environments, one-site adjoints, Jacobian)
    and checks E = e_core + h.gamma + 1/2 eri.Gamma against <psi|H|psi> from H_eff."""
    import numpy as np
    import torch
    from paper_2310_03920_gb300 import b2
    from synth import ab_initio_integrals
    n, N, M = 24, 24, 500
    h, eri = ab_initio_integrals(n, seed=24)
    ctx = b2.Context(0)
    mpo = b2.b2_build_mpo(ctx, h, eri, 0.0, N, 0)
    mps = b2.b2_mps_random(ctx, mpo, M, seed=124)
    b2.b2_rdm_grad(ctx, mpo, mps, n)                # warm-up (kernel attributes, allocator)
    times = []
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g1, g2 = b2.b2_rdm_grad(ctx, mpo, mps, n)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    env = b2.b2_env_init(ctx, mpo, mps, 0)
    nel, _ = b2.b2_psi_layout(ctx, env, 0)
    psi = torch.empty(nel, dtype=torch.float64, device="cuda")
    out = torch.empty_like(psi)
    b2.b2_psi_from_mps(ctx, env, 0, psi)
    b2.b2_heff_apply(ctx, env, 0, psi, out)
    torch.cuda.synchronize()
    e_env = float(torch.dot(psi, out) / torch.dot(psi, psi))
    e_rdm = float(np.sum(h * g1) + np.sum(eri * g2))
    sec = float(np.median(times))
    line = {"metric": METRIC, "value": sec, "unit": "s per gradient", "n_gpus": 1,
            "steps": len(times), "warmup": 1, "ms_per_step": sec * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "abinitio_n24_N24_M500_rdm_gradient", "n": n, "n_elec": N, "M": M},
            "gradient_elements": n * n + n ** 4, "energy_identity_abs_err": abs(e_env - e_rdm),
            "trace_gamma": float(np.trace(g1))}
    print(json.dumps(line), flush=True)
    b2.b2_free_env(env)
    b2.b2_free_mps(mps)
    b2.b2_free_mpo(mpo)
    ctx.close()


def run_eig(args):
    """The truncation eigensolver alone (b2_eigh_batched): one batch shaped like a
    truncation step of the Hubbard L = 32, M = 500 sweep (43 sectors, dims 147 .. 2) of
    graded density-matrix-like matrices (synth.graded_density_matrices, seed 5).  value =
    applied-rotation flops (12 m_active + 6 m per rotation) / device time of the batched call."""
    import numpy as np
    import torch
    from paper_2310_03920_gb300 import b2
    from synth import TRUNCATION_BATCH_DIMS, graded_density_matrices
    dims = TRUNCATION_BATCH_DIMS
    mats = graded_density_matrices(dims, seed=5)
    a = torch.tensor(np.concatenate([x.ravel() for x in mats]), device="cuda")
    ev = torch.empty(sum(dims), dtype=torch.float64, device="cuda")
    vec = torch.empty(sum(d * d for d in dims), dtype=torch.float64, device="cuda")
    ctx = b2.Context(0)
    for _ in range(args.warmup):
        b2.b2_eigh_batched(ctx, dims, a, ev, vec)
    torch.cuda.synchronize()
    b2.b2_profile(ctx, True)
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            b2.b2_eigh_batched(ctx, dims, a, ev, vec)
        torch.cuda.synchronize()
    prof = b2.b2_profile_read(ctx)
    b2.b2_profile(ctx, False)
    v = vec[:dims[0] ** 2].cpu().numpy().reshape(dims[0], dims[0])
    w = ev[:dims[0]].cpu().numpy()
    resid = float(np.abs(mats[0] @ v - v * w).max())
    ms = prof["eig_ms"] / max(1, args.steps)
    ach = prof["eig_flops"] / (prof["eig_ms"] * 1e-3) / 1e12 if prof["eig_ms"] > 0 else 0.0
    peak = measured_peaks(torch)["fp64_tflops_measured"]
    line = {"metric": METRIC, "value": ach, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "truncation_batch43_graded_density_matrices", "dims": dims,
                       "spectrum": "10^(-16 i/(r-1)), r = 0.7 m + 1, zero beyond",
                       "l2": "inputs resident (~1.2 MB); the kernel works in L2"},
            "roofline": {"kernel": "k_jacobi + k_jacobi_cluster (12 m_active + 6 m flops per applied rotation)",
                         "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak if peak else None,
                         "peak_source": "measured cuBLAS DGEMM 8192^3 on this GPU (FP64)",
                         "traffic": None},
            "residual_largest": resid, "gpu_launches": int(prof["launches"]),
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    args = parse()
    rank, world, local = dist_info()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch64":
        run_batch(args)
        return
    if args.workload == "batch64_sweeps":
        run_batch_sweeps(args)
        return
    if args.workload == "grad_n24":
        run_grad(args)
        return
    if args.workload == "eig_batch":
        run_eig(args)
        return
    if args.workload == "sweep_n36":
        run_sweep_n36(args)
        return
    if args.workload != "sweep":
        run_window(args)
        return
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2310_03920_gb300 import b2

    prec = b2.PRECISIONS[args.prec]
    h, eri, bonds, sites = workload_inputs()
    L, M = WORKLOAD["L"], WORKLOAD["M"]
    ctx = b2.Context(local)
    mpo_h = b2.b2_build_mpo(ctx, h, eri, 0.0, L, 0)
    mps_h = b2.b2_mps_import(ctx, bonds, sites, L, 0, center=0)
    env_h = b2.b2_env_init(ctx, mpo_h, mps_h, center=0)
    # setup sweeps (untimed): bonds grow to M, the energy settles (1e-10) and at least four
    # sweeps run at the full bond dimension, so that the density matrices have stopped
    # rotating and the eigensolver's warm start is in its steady state
    settle = []
    t_settle = time.perf_counter()
    for _ in range(18):
        r = b2.b2_sweep(ctx, mpo_h, mps_h, env_h, [M], prec=prec)[0]
        settle.append(r)
        at_m = sum(x["max_bond"] >= M for x in settle)
        if (at_m >= 4 and len(settle) > 1
                and abs(r["energy"] - settle[-2]["energy"]) < 1e-10):
            break
    t_settle = time.perf_counter() - t_settle
    # warm-up sweeps
    for _ in range(args.warmup):
        b2.b2_sweep(ctx, mpo_h, mps_h, env_h, [M], prec=prec)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    energies, flops, step_ms, breakdown = [], 0.0, [], []
    b2.b2_profile(ctx, True)
    barrier()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)                       # L2 flushed between steps (256 MB write)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            # profiler range = the timed sweeps (for ncu --profile-from-start off)
            torch.cuda.cudart().cudaProfilerStart()
            e0.record(stream)
            res = b2.b2_sweep(ctx, mpo_h, mps_h, env_h, [M], prec=prec)
            e1.record(stream)
            torch.cuda.synchronize()
            torch.cuda.cudart().cudaProfilerStop()
            step_ms.append(e0.elapsed_time(e1))
            energies.append(res[0]["energy"])
            flops += res[0]["matvec_flops"]
            breakdown.append({k: res[0][k] for k in ("t_davidson", "t_split", "n_matvec",
                                                     "discarded_weight", "max_bond")})
    barrier()
    prof = b2.b2_profile_read(ctx)
    b2.b2_profile(ctx, False)
    t_step = sum(step_ms) / len(step_ms)
    t_tot = sum(step_ms) * 1e-3
    t_tot, flops_all = aggregate_ranks(t_tot, flops, "cuda")
    value = flops_all / t_tot / 1e12

    # e2e through the public API from host buffers: import, env, one sweep, export
    bonds_now, sites_now, _ = b2.b2_mps_export(ctx, mps_h)
    h2d = sum(b.nbytes for blocks in sites_now for b in blocks.values())
    e2e_ms, e2e_flops, d2h = [], 0.0, 0
    for _ in range(0 if args.no_e2e else max(1, min(args.steps, 2))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = b2.b2_mps_import(ctx, bonds_now, sites_now, L, 0, center=0)
        en2 = b2.b2_env_init(ctx, mpo_h, s2, center=0)
        r2 = b2.b2_sweep(ctx, mpo_h, s2, en2, [M], prec=prec)
        out = b2.b2_mps_export(ctx, s2)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e2e_flops += r2[0]["matvec_flops"]
        d2h = sum(b.nbytes for blocks in out[1] for b in blocks.values())
        b2.b2_free_env(en2)
        b2.b2_free_mps(s2)
    e2e_val = e2e_flops / (sum(e2e_ms) * 1e-3) / 1e12 if e2e_ms else None

    # mixed precision vs FP64 on the same state: one sweep each from the MPS after the timed
    # sweeps (split precision with FP64 refinement to the same |r|^2 threshold)
    mixed = None
    if args.prec == "fp64" and not args.no_mixed:
        mixed = {}
        for name, pr in (("fp64", b2.B2_FP64), ("bf16x3", b2.B2_BF16X3), ("tf32x3", b2.B2_TF32X3)):
            s3 = b2.b2_mps_import(ctx, bonds_now, sites_now, L, 0, center=0)
            en3 = b2.b2_env_init(ctx, mpo_h, s3, center=0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r3 = b2.b2_sweep(ctx, mpo_h, s3, en3, [M], prec=pr)
            torch.cuda.synchronize()
            mixed[name] = {"sweep_ms": (time.perf_counter() - t0) * 1e3,
                           "energy": r3[0]["energy"], "n_matvec": r3[0]["n_matvec"]}
            b2.b2_free_env(en3)
            b2.b2_free_mps(s3)
        for name in ("bf16x3", "tf32x3"):
            mixed[name]["dE_vs_fp64"] = abs(mixed[name]["energy"] - mixed["fp64"]["energy"])
            mixed[name]["speedup_vs_fp64"] = mixed["fp64"]["sweep_ms"] / mixed[name]["sweep_ms"]

    # sweep variants from the same state (FP64): the one-site sweep, a two-site sweep with
    # perturbative noise and a three-root state-averaged sweep; two sweeps each, the second
    # timed (eigensolver warm-start cache and window programs in place, as in the main line)
    variants = None
    if args.prec == "fp64" and not args.no_mixed:
        variants = {}
        for name, kw in (("two_site", {}), ("one_site", {"dots": [1, 1]}),
                         ("two_site_noise_1e-5", {"noise": [1e-5, 1e-5]}),
                         ("state_average_3roots", {"n_roots": 3, "dav_max_iter": 200,
                                                   "max_subspace": 40})):
            s3 = b2.b2_mps_import(ctx, bonds_now, sites_now, L, 0, center=0)
            en3 = b2.b2_env_init(ctx, mpo_h, s3, center=0)
            b2.b2_sweep(ctx, mpo_h, s3, en3, [M], **{k: (v[:1] if isinstance(v, list) else v)
                                                    for k, v in kw.items()})
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r3 = b2.b2_sweep(ctx, mpo_h, s3, en3, [M], **{k: (v[1:] if isinstance(v, list) else v)
                                                         for k, v in kw.items()})[0]
            torch.cuda.synchronize()
            variants[name] = {"sweep_ms": (time.perf_counter() - t0) * 1e3,
                              "energy": r3["energy"], "n_matvec": r3["n_matvec"],
                              "max_bond": r3["max_bond"],
                              "t_davidson_ms": r3["t_davidson"] * 1e3,
                              "t_split_ms": r3["t_split"] * 1e3}
            if "n_roots" in kw:
                variants[name]["root_energy"] = r3["root_energy"]
            b2.b2_free_env(en3)
            b2.b2_free_mps(s3)

    if rank != 0:
        return
    peaks = measured_peaks(torch)
    fp64_peak = peaks["fp64_tflops_measured"]
    # DRAM bytes per launch from ncu captures of this sweep (dram__bytes_read.sum +
    # dram__bytes_write.sum of the launches of one timed sweep): an eigensolver call = 192/61
    # cluster launches of 0.35 MB + one one-CTA launch of 0.07 MB; k_gemm 1.35 MB (120
    # launches of the register-staged quadrant kernel)
    traffic = {"eig": 192.0 / 61.0 * 0.35e6 + 0.07e6, "k_gemm": 1.35e6}

    def fp64_roofline(kernel, flops_, ms_, launches_, traffic_=None):
        ach = flops_ / (ms_ * 1e-3) / 1e12 if ms_ > 0 else 0.0
        return {"kernel": kernel, "bound": "alu", "achieved": ach, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": ach / fp64_peak if fp64_peak else None,
                "peak_source": "measured cuBLAS DGEMM 8192^3 on this GPU (FP64; not in "
                               "MEASURED_PEAKS.json)",
                "launches": launches_, "avg_launch_us": ms_ * 1e3 / max(1, launches_),
                "device_ms_per_step": ms_ / max(1, args.steps), "traffic": traffic_,
                "traffic_unit": "bytes per launch (ncu capture of this workload)"}

    # the dominant kernel of the sweep (by device time) is reported as "roofline"
    rl_heff = fp64_roofline("k_gemm (H_eff block contraction, FP64)", prof["heff_flops"],
                            prof["heff_ms"], prof["heff_launches"], traffic["k_gemm"])
    rl_eig = fp64_roofline("k_jacobi + k_jacobi_cluster (truncation eigensolver, FP64; "
                           "12 m_active + 6 m flops per applied rotation of an m x m block)",
                           prof["eig_flops"], prof["eig_ms"], prof["eig_launches"], traffic["eig"])
    if prof["eig_ms"] > prof["heff_ms"]:
        roofline, roofline_other = rl_eig, rl_heff
    else:
        roofline, roofline_other = rl_heff, rl_eig
    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.prec == "fp64" else args.prec, "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "L": L, "t": WORKLOAD["t"], "U": WORKLOAD["U"],
                       "n_elec": L, "two_sz": 0, "M": M, "prec": args.prec,
                       "l2": "flushed between steps (256 MB write)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "setup_sweeps": {"count": len(settle), "seconds": t_settle,
                             "energies": [r["energy"] for r in settle],
                             "max_bond": [r["max_bond"] for r in settle]},
            "sweep_energy": energies[-1], "sweep_ms": step_ms, "sweep_breakdown": breakdown,
            "roofline": roofline, "roofline_other": roofline_other,
            "device_ms_per_step": {"heff_contraction": prof["heff_ms"] / args.steps,
                                   "truncation_eigensolver": prof["eig_ms"] / args.steps,
                                   "davidson_rayleigh_ritz": prof["rr_ms"] / args.steps},
            "gpu_launches": int(prof["launches"]),
            "clocks": clk.summary(),
            "e2e": {"value": e2e_val, "unit": "TFLOP/s",
                    "ms_per_step": statistics.mean(e2e_ms) if e2e_ms else None,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}}
    if mixed is not None:
        line["mixed_vs_fp64_sweep"] = mixed
    if variants is not None:
        line["sweep_variants"] = variants
    # the reference arm's sample on the GPU: FP64 products at the same window of the same
    # random MPS (like-for-like with the oracle's milliseconds per product)
    ms_p, fl_p = gpu_middle_window_product(b2, torch, ctx)
    line["middle_window_product"] = {"ms": ms_p, "library_flops": fl_p,
                                     "tflops": fl_p / (ms_p * 1e-3) / 1e12,
                                     "input": "window (15, 16) of the workload's random MPS"}
    if not args.no_window:
        b2.b2_profile(ctx, True)
        line["abinitio_n36_window"] = {
            "M1000": window_leg(b2, torch, ctx, 1000, True, 3, peaks),
            "M2000": window_leg(b2, torch, ctx, 2000, False, 3, peaks)}
        b2.b2_profile(ctx, False)
    if not args.no_cpu_baseline and world == 1:
        budget = args.cpu_budget
        sec, nprod, setup, fl = oracle_sample(budget)
        c = WORKLOAD["L"] // 2 - 1
        line["cpu_baseline"] = {"value": fl / sec / 1e12, "unit": "TFLOP/s", "cores": cpu_cores(),
                                "kind": "oracle",
                                "sample": "%d oracle H_eff.psi products at the middle window "
                                          "(sites %d, %d) of the workload's random MPS (setup "
                                          "%.1f s, %.1f ms per product; flops counted by the "
                                          "oracle)" % (nprod, c, c + 1, setup, sec * 1e3)}
    print(json.dumps(line), flush=True)
    b2.b2_free_env(env_h)
    b2.b2_free_mps(mps_h)
    b2.b2_free_mpo(mpo_h)
    ctx.close()


if __name__ == "__main__":
    main()
