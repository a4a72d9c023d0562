"""Benchmark: HBMC-ICCG time to a 1e-8 relative residual on one GB300.

Workload (default): 3D 7-point Poisson on a 128^3 grid (2,097,152 unknowns,
14,581,760 nonzeros, Dirichlet, natural order), BMC blocks = 2x2x2 boxes
(bs = 8), w = 32, greedy block coloring (2 colors), b = A x* with
x* ~ U(-1, 1), x0 = 0, tolerance 1e-8.  A step is one complete hbmc_iccg
call: permute b in, the CG loop with both substitutions, permute x out and
the true residual; the IC(0) factorization is timed separately.

The line also carries, under "configs", the other configurations in the
launch configuration the library picks for them (skip with --no-configs):
the heterogeneous 27-point 96^3 and 3-DOF vector-Laplacian 100^3 systems in
a random order with FP32 substitutions (time, iterations, residual, per-sweep
bandwidth), the 256-system batch (autotuned, aggregate bandwidth, per-system
times) and the learned IC shift (trained on the GPU from shift sweeps,
held-out gain over the plain rule, and its use on those configurations and
on an IEEJ-sized curl-curl system).

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on
the host cores instead (each step a bounded sample of the same solve: the
start of the solve plus a few PCG iterations, extrapolated to the full
iteration count).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ICCG time to 1e-8 FP64 residual; fwd/bwd subst GB/s vs HBM roofline"
TOL = 1e-8
GRID = 128
DEFAULT_BS = 8


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------

def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def init_dist(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist if world > 1 else None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value, device="cpu"):
    """Max of a float over all ranks (identity on one rank)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


TRAFFIC_RECORD = os.path.join("profiles", "spmv_tma_poisson128_bs8_f64.md")
SPMV_SOURCE = os.path.join("paper_1908_00741_gb300", "csrc", "spmv_tma.cu")


def measured_traffic():
    """DRAM bytes per launch of the SpMV kernel from the committed ncu summary
    (its `traffic:` line), or None when the kernel source changed since the
    counters were taken (the line carries the source's sha1)."""
    import hashlib
    import re
    try:
        text = open(os.path.join(ROOT, TRAFFIC_RECORD)).read()
        m = re.search(r"traffic: kernel=(\S+) bytes_per_launch=(\d+) source=(\S+) sha1=([0-9a-f]+)", text)
        sha = hashlib.sha1(open(os.path.join(ROOT, m.group(3)), "rb").read()).hexdigest()
        return int(m.group(2)) if sha == m.group(4) else None
    except Exception:
        return None


# Nominal FP64 rate of a GB300 (1.25 TFLOP/s dense): the ceiling for the
# FP64 fused multiply-adds every kernel of the FP64 path issues.
FP64_NOMINAL_TFLOPS = 1.25


# The roofline the scope statement names: bytes over 8 TB/s (nominal HBM3e).
# Every fraction is also given against the measured copy bandwidth.
HBM_NOMINAL_GBS = 8000.0


def host_info():
    """This host's core count and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() == "Model name":
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part", "hardware")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            model = "unknown"
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


def fracs(gbs, peak):
    return {"frac": round(gbs / peak, 4), "frac_nominal": round(gbs / HBM_NOMINAL_GBS, 4)}


def subst_bytes(n, nnz_lower, s):
    """Algorithmic bytes of one forward / backward substitution (compulsory
    traffic: each nonzero of L once with its int32 column, dinv, the input
    vector in and the result out; the backward sweep also reads r for the
    fused r.z).  s = bytes per factor value."""
    fwd = nnz_lower * (s + 4) + n * s + n * 8 + n * s
    bwd = nnz_lower * (s + 4) + n * s + n * s + n * 8 + n * 8
    return fwd, bwd


def spmv_bytes(n, nnz):
    return nnz * 12 + 2 * n * 8


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

def run_gpu(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    from paper_1908_00741_gb300 import hbmc as H
    from paper_1908_00741_gb300 import workloads as W

    H.load()
    bs = args.bs
    P = W.poisson_problem(GRID, bs=bs)
    A = P.A
    prec = H.PREC_F32 if args.precision == "f32" else H.PREC_F64
    t0 = time.perf_counter()
    loop = H.LOOP_HOST if args.loop == "host" else H.LOOP_GRAPH
    ctx = H.hbmc_build(A, bs, 32, box=P.box, precision=prec, device=local, loop_mode=loop)
    build_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    H.hbmc_set_stream(ctx, stream)
    b = torch.tensor(P.b, device="cuda")
    x = torch.zeros_like(b)

    # IC(0): warm then time
    H.hbmc_ic0(ctx, 0.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st, bad = H.hbmc_ic0(ctx, 0.0)
    e1.record(stream)
    torch.cuda.synchronize()
    assert st == H.OK, bad
    ic0_ms = e0.elapsed_time(e1)

    def step():
        x.zero_()
        return H.hbmc_iccg(ctx, b, x, tol=TOL, maxit=10000)

    for _ in range(args.warmup):
        res = step()
    assert res.status == H.OK, res
    launches = ctx.info()["last_launches"]

    torch.cuda.synchronize()
    barrier(dist)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        total_launches = 0
        for _ in range(args.steps):
            res = step()
            total_launches += ctx.info()["last_launches"]
        ev[1].record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    torch.cuda.synchronize()
    ms_total = ev[0].elapsed_time(ev[1])
    ms_step = max_over_ranks(dist, ms_total / args.steps, "cuda")
    iters = res.iters
    true_relres = res.true_relres
    err = float(np.max(np.abs(x.cpu().numpy() - P.x_star)) / np.max(np.abs(P.x_star)))

    # e2e: same solve through the host-buffer entry point (H2D of b and x0,
    # D2H of x inside the timed region), pinned host memory
    bh = torch.tensor(P.b).pin_memory().numpy()
    xh = torch.zeros(A.n, dtype=torch.float64).pin_memory().numpy()
    for _ in range(2):
        xh[:] = 0.0
        H.hbmc_iccg_host(ctx, bh, xh, tol=TOL)
    torch.cuda.synchronize()
    e2e = []
    for _ in range(max(3, args.steps // 2)):
        xh[:] = 0.0
        t = time.perf_counter()
        H.hbmc_iccg_host(ctx, bh, xh, tol=TOL)
        e2e.append((time.perf_counter() - t) * 1e3)
    e2e_ms = max_over_ranks(dist, statistics.median(e2e), "cuda")

    # Per-phase device times of one CG iteration, CUDA events on this stream
    # around `reps` back-to-back runs of the same kernels the solve runs
    # (hbmc_profile_kernels), for the roofline figures.
    inf = ctx.info()
    nnz_l = inf["nnz_lower"]
    kernel_ms = {}
    for pname, pv in (("f64", H.PREC_F64), ("f32", H.PREC_F32)):
        H.hbmc_set_precision(ctx, pv)
        x.zero_()
        H.hbmc_iccg(ctx, b, x, tol=TOL)
        prof = H.hbmc_profile_kernels(ctx, 30)
        kernel_ms[f"fwd_{pname}"] = prof["fwd"]
        kernel_ms[f"bwd_{pname}"] = prof["bwd"]
        if pv == prec:
            kernel_ms["spmv"] = prof["spmv"]
            kernel_ms["update_xr"] = prof["update_xr"]
            kernel_ms["update_p"] = prof["update_p"]
    H.hbmc_set_precision(ctx, prec)

    peak, peak_kind = measured_peaks()
    gbs = {}
    for pname, s in (("f64", 8), ("f32", 4)):
        fb, bb = subst_bytes(A.n, nnz_l, s)
        gbs[f"fwd_{pname}"] = fb / (kernel_ms[f"fwd_{pname}"] * 1e-3) / 1e9
        gbs[f"bwd_{pname}"] = bb / (kernel_ms[f"bwd_{pname}"] * 1e-3) / 1e9
    sp_bytes = spmv_bytes(A.n, A.nnz)
    gbs["spmv"] = sp_bytes / (kernel_ms["spmv"] * 1e-3) / 1e9
    gbs["update_xr"] = 6 * A.n * 8 / (kernel_ms["update_xr"] * 1e-3) / 1e9
    gbs["update_p"] = 3 * A.n * 8 / (kernel_ms["update_p"] * 1e-3) / 1e9

    # dominant kernel of a solve: SpMV (the largest share in the launch list)
    traffic = measured_traffic()
    sp_fma = A.nnz + A.n  # q = A p plus the fused p.q
    sp_tflops = 2 * sp_fma / (kernel_ms["spmv"] * 1e-3) / 1e12
    roofline = {"bound": "hbm", "kernel": "k_spmv_tma (q = A p, fused p.q)", "achieved": round(gbs["spmv"], 1),
                "peak": peak, "unit": "GB/s", "frac": round(gbs["spmv"] / peak, 4),
                "traffic": traffic, "algorithmic_bytes": sp_bytes, "peak_source": peak_kind,
                "fp64": {"fma_per_launch": sp_fma, "achieved_tflops": round(sp_tflops, 4),
                         "peak_tflops": FP64_NOMINAL_TFLOPS, "frac": round(sp_tflops / FP64_NOMINAL_TFLOPS, 4),
                         "peak_source": "nominal"}}
    roofline.update({"frac_nominal": round(gbs["spmv"] / HBM_NOMINAL_GBS, 4), "peak_nominal": HBM_NOMINAL_GBS})
    subst = {k: {"GB/s": round(v, 1), **fracs(v, peak), "ms": round(kernel_ms[k], 4)} for k, v in gbs.items()}

    variants = {}
    if not args.no_variants:
        # the 32^3 configuration (32,768 unknowns, bs 8, FP64): it sits in L2, so time only
        P1 = W.poisson_problem(32, bs=8)
        c1 = H.hbmc_build(P1.A, 8, 32, box=P1.box, device=local)
        H.hbmc_set_stream(c1, stream)
        H.hbmc_ic0(c1)
        b1 = torch.tensor(P1.b, device="cuda")
        x1 = torch.zeros_like(b1)
        for _ in range(3):
            x1.zero_()
            r1 = H.hbmc_iccg(c1, b1, x1, tol=TOL)
        a1, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a1.record(stream)
        for _ in range(10):
            x1.zero_()
            r1 = H.hbmc_iccg(c1, b1, x1, tol=TOL)
        e1.record(stream)
        torch.cuda.synchronize()
        variants["poisson32_bs8_f64"] = {"ms": round(a1.elapsed_time(e1) / 10, 3), "iters": r1.iters,
                                         "true_relres": r1.true_relres}
        c1.close()
        for vbs in (8, 16, 32):
            for vp in ("f64", "f32"):
                if vbs == bs and vp == args.precision:
                    continue
                Pv = W.poisson_problem(GRID, bs=vbs) if vbs != bs else P
                cv = H.hbmc_build(Pv.A, vbs, 32, box=Pv.box, device=local,
                                  precision=H.PREC_F32 if vp == "f32" else H.PREC_F64)
                H.hbmc_set_stream(cv, stream)
                H.hbmc_ic0(cv)
                bv = torch.tensor(Pv.b, device="cuda")
                xv = torch.zeros_like(bv)
                for _ in range(2):
                    xv.zero_()
                    rv = H.hbmc_iccg(cv, bv, xv, tol=TOL)
                a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                reps = 5
                a.record(stream)
                for _ in range(reps):
                    xv.zero_()
                    rv = H.hbmc_iccg(cv, bv, xv, tol=TOL)
                c.record(stream)
                torch.cuda.synchronize()
                variants[f"bs{vbs}_{vp}"] = {"ms": round(a.elapsed_time(c) / reps, 3), "iters": rv.iters,
                                            "true_relres": rv.true_relres}
                cv.close()

    configs = {}
    if not args.no_configs:
        # the other configurations, each in the launch configuration the
        # library picks for it (FP32 substitutions in FP64 CG, as specified)
        cpu_it = args.cpu_config_iters if rank == 0 and world == 1 and not args.no_cpu_baseline else 0
        configs["hetero27_96_f32"] = config_solve(W.heterogeneous27_problem(args.hetero_m), H.PREC_F32, local,
                                                  stream, peak, "heterogeneous 27-point 96^3, random order",
                                                  cpu_iters=cpu_it)
        configs["veclap_100_f32"] = config_solve(W.vector_laplacian_problem(args.veclap_m), H.PREC_F32, local,
                                                 stream, peak, "3-DOF vector Laplacian 100^3 nodes, random order",
                                                 cpu_iters=cpu_it)
        configs["batch256_f32"] = batch_report(args, local, peak)
        configs["learned_shift"] = learned_report(args, local)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(P, iters, args.cpu_sample_iters)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": round(ms_step, 4), "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": args.precision, "data": "synthetic",
        "config": {"workload": f"7-point Poisson {GRID}^3 ({A.n} unknowns, {A.nnz} nonzeros), "
                               f"bs={bs} ({'x'.join(map(str, P.box))} boxes), w=32, "
                               f"FP{args.precision[1:]} substitutions, tol {TOL:g}",
                   "n": A.n, "nnz": A.nnz, "bs": bs, "w": 32, "colors": inf["nc"],
                   "precision": args.precision, "parallelism": f"replicas{world}", "loop": args.loop,
                   "l2": "inputs larger than L2 (device working set "
                         f"{inf['device_bytes'] / 1e9:.2f} GB)"},
        "iters": iters, "true_relres": true_relres, "max_rel_err_vs_xstar": err,
        "ic0_ms": round(ic0_ms, 3), "build_s": round(build_s, 3),
        "ms_per_iter": round(ms_step / max(iters, 1), 4),
        "e2e": {"value": round(e2e_ms, 4), "unit": "ms", "h2d_bytes_per_step": 2 * A.n * 8,
                "d2h_bytes_per_step": A.n * 8},
        "gpu_launches": int(total_launches), "launches_per_step": int(launches),
        "roofline": roofline, "subst_roofline": subst, "variants": variants, "configs": configs,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(P, gpu_iters, sample_iters, what="the 128^3 solve"):
    """The oracle as it stands: single-threaded FP64 C, on this host.  Sample:
    setup (blocking, coloring, reordering, IC(0)) plus `sample_iters` PCG
    iterations; value = setup-free solve time scaled to the GPU's iteration
    count."""
    import oracle
    t = time.perf_counter()
    an = oracle.analyse(P.A, P.bs, P.w, box=P.box)
    lval, _, dinv, bad = oracle.factor(an, 0.0)
    setup_s = time.perf_counter() - t
    t = time.perf_counter()
    oracle.pcg(an, lval, dinv, P.b, tol=TOL, maxit=0)
    start_s = time.perf_counter() - t
    t = time.perf_counter()
    s = oracle.pcg(an, lval, dinv, P.b, tol=TOL, maxit=sample_iters)
    dt = time.perf_counter() - t
    per_iter = max(dt - start_s, 0.0) / max(s.iters, 1)
    return {"value": round((start_s + per_iter * gpu_iters) * 1e3, 3), "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": f"the start and {s.iters} PCG iterations of {what} ({dt:.2f} s, + {setup_s:.2f} s "
                      f"setup not counted); value = start + per-iteration time x {gpu_iters} iterations",
            "scaled_from_iters": int(s.iters), "sample_s": round(dt, 3), "host": host_info()}


def config_solve(P, prec, local, stream, peak, name, reps=5, loop=None, cpu_iters=0):
    """One configuration: solve time (CUDA events, inputs resident), CG
    iterations, true residual, and the per-sweep device times with their
    algorithmic bandwidth against the measured and the nominal HBM peak."""
    import torch
    from paper_1908_00741_gb300 import hbmc as H
    t = time.perf_counter()
    ctx = H.hbmc_build(P.A, P.bs, 32, box=P.box, precision=prec, device=local,
                       loop_mode=H.LOOP_GRAPH if loop is None else loop)
    build_s = time.perf_counter() - t
    H.hbmc_set_stream(ctx, stream)
    st, bad = H.hbmc_ic0(ctx)
    assert st == H.OK, bad
    b = torch.tensor(P.b, device="cuda")
    x = torch.zeros_like(b)
    for _ in range(2):
        x.zero_()
        res = H.hbmc_iccg(ctx, b, x, tol=TOL)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(reps):
        x.zero_()
        res = H.hbmc_iccg(ctx, b, x, tol=TOL)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / reps
    prof = H.hbmc_profile_kernels(ctx, 20)
    inf = ctx.info()
    s = 4 if prec == H.PREC_F32 else 8
    fb, bb = subst_bytes(P.A.n, inf["nnz_lower"], s)
    fwd_gbs = fb / (prof["fwd"] * 1e-3) / 1e9
    bwd_gbs = bb / (prof["bwd"] * 1e-3) / 1e9
    sp_gbs = spmv_bytes(P.A.n, P.A.nnz) / (prof["spmv"] * 1e-3) / 1e9
    out = {"workload": name, "n": P.A.n, "nnz": P.A.nnz, "bs": P.bs, "w": 32, "colors": inf["nc"],
           "precision": "f32" if s == 4 else "f64", "ms": round(ms, 3), "iters": res.iters,
           "status": res.status, "true_relres": res.true_relres, "ms_per_iter": round(ms / max(res.iters, 1), 4),
           "build_s": round(build_s, 2), "launches_per_solve": inf["last_launches"],
           "subst_roofline": {
               "fwd": {"ms": round(prof["fwd"], 4), "GB/s": round(fwd_gbs, 1), **fracs(fwd_gbs, peak)},
               "bwd": {"ms": round(prof["bwd"], 4), "GB/s": round(bwd_gbs, 1), **fracs(bwd_gbs, peak)},
               "spmv": {"ms": round(prof["spmv"], 4), "GB/s": round(sp_gbs, 1), **fracs(sp_gbs, peak)}}}
    ctx.close()
    if cpu_iters > 0:  # the oracle beside it, FP64 throughout, on a bounded sample
        out["cpu_baseline"] = cpu_baseline(P, res.iters, cpu_iters, what=f"the {name} solve")
    return out


def run_config(args):
    """One of the random-order configurations on its own (config3: the
    heterogeneous 27-point 96^3 system; config5: the 3-DOF vector Laplacian
    100^3), FP32 substitutions: the line the default run carries under
    "configs", with the clocks of its own timed region."""
    import torch
    from paper_1908_00741_gb300 import hbmc as H
    from paper_1908_00741_gb300 import workloads as W
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    peak, _ = measured_peaks()
    P, name = ((W.heterogeneous27_problem(args.hetero_m), f"heterogeneous 27-point {args.hetero_m}^3, random order")
               if args.workload == "config3" else
               (W.vector_laplacian_problem(args.veclap_m), f"3-DOF vector Laplacian {args.veclap_m}^3 nodes, "
                                                           "random order"))
    prec = H.PREC_F64 if args.precision == "f64" else H.PREC_F32
    with ClockSampler(local) as clk:
        rep = config_solve(P, prec, local, torch.cuda.current_stream(), peak, name, reps=args.steps,
                           loop=H.LOOP_HOST if args.loop == "host" else H.LOOP_GRAPH)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.cpu_config_iters > 0:
        # outside the clock window: the GPU idles meanwhile
        rep["cpu_baseline"] = cpu_baseline(P, rep["iters"], args.cpu_config_iters, what=f"the {name} solve")
    line = {"metric": METRIC, "value": rep["ms"], "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rep["ms"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": rep["precision"], "data": "synthetic",
            "config": {k: rep[k] for k in ("workload", "n", "nnz", "bs", "w", "colors", "precision")},
            **{k: v for k, v in rep.items() if k not in ("workload", "ms")}, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# batched workload: 256 uneven systems
# --------------------------------------------------------------------------

def batch_report(args, local, peak, steps=3, warmup=2):
    """The 256-system batch (FP32 substitutions, FP64 CG): autotuned on a
    32-system subset, then solved together.  Aggregate algorithmic bandwidth:
    every system's per-iteration bytes (SpMV, both FP32 substitutions, nine
    vector passes) times its iterations, over the batch's solve time."""
    import torch
    from paper_1908_00741_gb300 import hbmc as H
    from paper_1908_00741_gb300 import workloads as W
    t = time.perf_counter()
    items = W.batch_problems(args.batch_systems)
    gen_s = time.perf_counter() - t
    mats = [A for A, _, _ in items]
    bvec = np.concatenate([b for _, b, _ in items])
    n_total = int(sum(A.n for A in mats))
    sub = mats[:32]
    bsub = torch.tensor(np.concatenate([b for _, b, _ in items[:32]]), device="cuda")
    t = time.perf_counter()
    bs_cand, w_cand, v_cand = (4, 8, 16, 32), (16, 32), (0, 8)
    best, best_w, best_v, cand_ms = H.hbmc_batch_autotune_w(sub, bsub, bs_cand, w_cand, v_cand,
                                                            precision=H.PREC_F32, tol=TOL)
    tune_s = time.perf_counter() - t
    t = time.perf_counter()
    batch = H.hbmc_batch_build(mats, best, w=best_w, vslice=best_v, precision=H.PREC_F32, device=local)
    build_s = time.perf_counter() - t
    stream = torch.cuda.current_stream()
    H.hbmc_batch_set_stream(batch, stream)
    st, bad = H.hbmc_batch_ic0(batch)
    assert st == H.OK
    b = torch.tensor(bvec, device="cuda")
    x = torch.zeros_like(b)
    for _ in range(warmup):
        x.zero_()
        res = H.hbmc_batch_iccg(batch, b, x, tol=TOL)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(steps):
        x.zero_()
        res = H.hbmc_batch_iccg(batch, b, x, tol=TOL)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / steps
    inf = batch.info()
    per_iter = np.array([spmv_bytes(A.n, A.nnz) + sum(subst_bytes(A.n, (A.nnz - A.n) // 2, 4)) + 9 * A.n * 8
                         for A in mats], dtype=np.float64)
    gbs = float((per_iter * res.iters).sum() / (ms * 1e-3) / 1e9)
    batch.close()
    return {"workload": f"{len(mats)} systems, 7/27-point stencils n^3 with n in [16, 64], lognormal "
                        f"sigma in [0, 2], natural order, box blocking",
            "systems": len(mats), "n_total": n_total, "nnz_total": int(sum(A.nnz for A in mats)),
            "bs": best, "w": best_w, "vslice": best_v, "colors": inf["nc"], "units": inf["units"],
            "ms": round(ms, 3),
            "all_converged": bool(res.status == H.OK), "max_true_relres": float(res.true_relres.max()),
            "iters": {"min": int(res.iters.min()), "median": float(np.median(res.iters)),
                      "max": int(res.iters.max())},
            "per_system_ms": {"min": round(float(res.solve_ms.min()), 3),
                              "median": round(float(np.median(res.solve_ms)), 3),
                              "max": round(float(res.solve_ms.max()), 3)},
            "aggregate": {"GB/s": round(gbs, 1), **fracs(gbs, peak),
                          "unknowns_per_s": round(n_total / (ms * 1e-3), 1)},
            "autotune": {"subset": "the first 32 systems", "bs": list(bs_cand), "w": list(w_cand),
                         "vslice": list(v_cand),
                         "subset_ms": {f"bs{b}_w{w}_v{v}": round(float(cand_ms[i, j, k]), 3)
                                       for i, b in enumerate(bs_cand) for j, w in enumerate(w_cand)
                                       for k, v in enumerate(v_cand)},
                         "best_bs": best, "best_w": best_w, "best_vslice": best_v,
                         "slice_height": "w" if best_v == 0 else "per slice from {w, w/2, w/4}",
                         "seconds": round(tune_s, 2)},
            "gen_s": round(gen_s, 1), "build_s": round(build_s, 1)}

def run_batch(args):
    """256 independent SPD systems (7- or 27-point, n^3 with n ~ U{16..64},
    lognormal sigma ~ U[0, 2]) solved together; block size chosen by the
    library's autotuner on a 32-system subset; FP32 substitutions, FP64 CG."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    peak, _ = measured_peaks()
    with ClockSampler(local) as clk:
        rep = batch_report(args, local, peak, steps=args.steps, warmup=args.warmup)
    line = {"metric": "batched ICCG time to 1e-8 FP64 residual (all systems)", "value": rep["ms"], "unit": "ms",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": rep["ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32-subst/f64-cg",
            "data": "synthetic", "config": {k: rep[k] for k in ("workload", "systems", "n_total", "nnz_total",
                                                                 "bs", "w", "colors", "units")},
            **{k: v for k, v in rep.items() if k not in ("workload", "ms")}, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# learned IC shift: train on shift sweeps, then compare with the plain rule
# --------------------------------------------------------------------------

def learned_report(args, local):
    """Train the shift network on the GPU from shift sweeps over generated
    systems, compare it with the plain rule on held-out systems, and use it on
    the 27-point, 3-DOF and curl-curl configurations."""
    import torch
    from paper_1908_00741_gb300 import hbmc as H
    from paper_1908_00741_gb300 import learned_shift as LS
    from paper_1908_00741_gb300 import workloads as W

    t = time.perf_counter()
    train = W.learned_family(args.learned_train, 5000)
    held = W.learned_family(args.learned_heldout, 90000)
    gen_s = time.perf_counter() - t
    t = time.perf_counter()
    sw = LS.sweep([A for A, _ in train], [b for _, b in train], bs=8, maxit=3000)
    X, T = LS.dataset(sw)
    sweep_s = time.perf_counter() - t
    t = time.perf_counter()
    net = LS.train(X, T, steps=4000, lr=3e-3)
    train_s = time.perf_counter() - t
    swh = LS.sweep([A for A, _ in held], [b for _, b in held], bs=8, maxit=3000)
    plain, learned, best, fb = LS.evaluate(net, swh)

    def solve(P, name):
        ctx = H.hbmc_build(P.A, P.bs, 32, box=P.box, precision=H.PREC_F32, device=local)
        b = torch.tensor(P.b, device="cuda")
        rows = {}
        for tag, nn in (("plain_rule", None), ("learned", net)):
            st, shift, used_fb = H.hbmc_ic0_auto(ctx, nn)
            assert st == H.OK
            x = torch.zeros_like(b)
            H.hbmc_iccg(ctx, b, x, tol=TOL, maxit=20000)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record()
            reps = 3
            for _ in range(reps):
                x.zero_()
                r = H.hbmc_iccg(ctx, b, x, tol=TOL, maxit=20000)
            ev[1].record()
            torch.cuda.synchronize()
            rows[tag] = {"shift": shift, "fallback": used_fb, "iters": r.iters, "status": r.status,
                         "true_relres": r.true_relres, "ms": round(ev[0].elapsed_time(ev[1]) / reps, 3)}
        ctx.close()
        return {"workload": name, "n": P.A.n, "nnz": P.A.nnz, **rows}

    return {
        "family": "curl-curl systems (IC(0) needs a shift), 3-DOF vector Laplacians and heterogeneous "
                  "27-point stencils, random order",
        "train_systems": len(train), "heldout_systems": len(held), "shift_grid": list(H.shift_grid()),
        "heldout": {"plain_mean_iters": float(plain.mean()), "learned_mean_iters": float(learned.mean()),
                    "best_mean_iters": float(best.mean()), "gain_vs_plain": float(1 - learned.mean() / plain.mean()),
                    "fallbacks": int(fb.sum()), "systems": int(len(plain))},
        "training": {"samples": int(len(T)), "sweep_s": round(sweep_s, 1), "train_s": round(train_s, 2),
                     "gen_s": round(gen_s, 1)},
        "config5": solve(W.vector_laplacian_problem(args.veclap_m, bs=8),
                         f"3-DOF vector Laplacian {args.veclap_m}^3 nodes"),
        "config3": solve(W.heterogeneous27_problem(args.hetero_m, bs=8), f"heterogeneous 27-point {args.hetero_m}^3"),
        "curl_curl": solve(W.curl_curl_problem(args.curl_m),
                           f"curl-curl + 0.01 I on {args.curl_m}^3 cells (edge unknowns)"),
    }


def run_learned(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    rep = learned_report(args, local)
    line = {
        "metric": "CG iterations to 1e-8 with the learned IC shift vs the plain positive-pivot rule",
        "value": rep["heldout"]["learned_mean_iters"], "unit": "iterations (held-out mean)",
        "higher_is_better": False, "n_gpus": world, "dtype": "f32-subst/f64-cg", "data": "synthetic",
        "config": {"workload": rep["family"], "train_systems": rep["train_systems"],
                   "heldout_systems": rep["heldout_systems"], "shift_grid": rep["shift_grid"], "bs": 8, "w": 32},
        **{k: v for k, v in rep.items() if k not in ("family", "train_systems", "heldout_systems", "shift_grid")},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# reference arm: the CPU oracle
# --------------------------------------------------------------------------

def run_orderings(args):
    """The paper's comparison (Section 5, Tables "number-ite" and "Results")
    on the 128^3 7-point workload with the library's own kernels: MC = nodal
    multi-color ordering (blocks of one unknown, bs = 1, w = 32); BMC = block
    multi-color without the secondary reordering (bs = 8, w = 1: a level-1
    block is one BMC block, so pi_HBMC = pi_BMC); HBMC (bs = 8, w = 32).  FP64
    throughout; iterations, ms per solve and us per CG iteration."""
    import torch
    from paper_1908_00741_gb300 import hbmc as H
    from paper_1908_00741_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    rows = {}
    with ClockSampler(local) as clk:
        for name, bs, w in (("MC", 1, 32), ("BMC", 8, 1), ("HBMC", 8, 32)):
            P = W.poisson_problem(GRID, bs=bs)
            ctx = H.hbmc_build(P.A, bs, w, box=P.box, device=local)
            H.hbmc_set_stream(ctx, stream)
            assert H.hbmc_ic0(ctx)[0] == H.OK
            b = torch.tensor(P.b, device="cuda")
            x = torch.zeros_like(b)
            for _ in range(args.warmup):
                x.zero_()
                res = H.hbmc_iccg(ctx, b, x, tol=TOL, maxit=10000)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            for _ in range(args.steps):
                x.zero_()
                res = H.hbmc_iccg(ctx, b, x, tol=TOL, maxit=10000)
            ev[1].record(stream)
            torch.cuda.synchronize()
            ms = ev[0].elapsed_time(ev[1]) / args.steps
            inf = ctx.info()
            rows[name] = {"bs": bs, "w": w, "colors": inf["nc"], "iters": res.iters, "status": res.status,
                          "true_relres": res.true_relres, "ms": round(ms, 3),
                          "us_per_iter": round(ms * 1e3 / max(res.iters, 1), 1)}
            ctx.close()
    if rank != 0:
        return
    line = {
        "metric": "ICCG time to 1e-8 FP64 residual under MC, BMC and HBMC orderings", "value": rows["HBMC"]["ms"],
        "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": rows["HBMC"]["ms"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"7-point Poisson {GRID}^3, natural input order; MC bs=1 w=32, BMC bs=8 w=1, "
                               f"HBMC bs=8 w=32 (2x2x2 boxes)"},
        "orderings": rows, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_sor(args):
    """Symmetric SOR (SSOR) sweeps on the 128^3 7-point workload, HBMC order
    with bs = 8, w = 32 (the Gauss-Seidel/SOR use of the ordering, Section 2).
    A step is hbmc_sor with `--sor-sweeps` symmetric sweeps (omega 1.5);
    the metric is ms per symmetric sweep.  Algorithmic bytes of one
    half-sweep: nnz * 12 (columns and values) + 3 n * 8 (x in, b in, x out)."""
    import torch
    from paper_1908_00741_gb300 import hbmc as H
    from paper_1908_00741_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    P = W.poisson_problem(GRID, bs=DEFAULT_BS)
    ctx = H.hbmc_build(P.A, DEFAULT_BS, 32, box=P.box, device=local)
    stream = torch.cuda.current_stream()
    H.hbmc_set_stream(ctx, stream)
    b = torch.tensor(P.b, device="cuda")
    x = torch.zeros_like(b)
    sweeps, omega = args.sor_sweeps, 1.5
    for _ in range(args.warmup):
        x.zero_()
        rel = H.hbmc_sor(ctx, b, x, omega, sweeps, True)
    torch.cuda.synchronize()
    barrier(dist)
    with ClockSampler(local) as clk:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        for _ in range(args.steps):
            x.zero_()
            rel = H.hbmc_sor(ctx, b, x, omega, sweeps, True)
        ev[1].record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    ms_step = max_over_ranks(dist, ev[0].elapsed_time(ev[1]) / args.steps, "cuda")
    # kernel-only: the sweeps alone on reordered vectors
    n_pad = ctx.info()["n_pad"]
    bb = torch.zeros(n_pad, dtype=torch.float64, device="cuda")
    xb = torch.zeros_like(bb)
    H.hbmc_sor_bar(ctx, bb, xb, omega, 2, True)
    a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    a.record(stream)
    H.hbmc_sor_bar(ctx, bb, xb, omega, reps, True)
    c.record(stream)
    torch.cuda.synchronize()
    sweep_ms = a.elapsed_time(c) / reps
    half_bytes = P.A.nnz * 12 + 3 * P.A.n * 8
    peak, peak_kind = measured_peaks()
    gbs = 2 * half_bytes / (sweep_ms * 1e-3) / 1e9
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        an = oracle.analyse(P.A, DEFAULT_BS, 32, box=P.box)
        t = time.perf_counter()
        oracle.sor_solve(an, P.b, omega=omega, sweeps=2, symmetric=True)
        dt = (time.perf_counter() - t) / 2
        cpu = {"value": round(dt * 1e3, 3), "unit": "ms per symmetric sweep", "cores": 1, "kind": "oracle",
               "sample": "2 symmetric sweeps of the 128^3 system (orc_sor, one core)"}
    if rank != 0:
        return
    line = {
        "metric": "symmetric SOR sweep time on the HBMC ordering", "value": round(sweep_ms, 4),
        "unit": "ms per symmetric sweep", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"7-point Poisson {GRID}^3, bs={DEFAULT_BS} (2x2x2 boxes), w=32, omega {omega}, "
                               f"{sweeps} symmetric sweeps per step", "n": P.A.n, "nnz": P.A.nnz},
        "relres_after_step": rel,
        "roofline": {"bound": "hbm", "kernel": "k_sor (both halves of a symmetric sweep)",
                     "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
                     "traffic": None, "algorithmic_bytes": 2 * half_bytes, "peak_source": peak_kind},
        "e2e": {"value": round(ms_step, 4), "unit": "ms per step (permutations, sweeps, residual)",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "clocks": clk.summary(), "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def run_ilu(args):
    """ILU(0)-preconditioned BiCGStab on the nonsymmetric 7-point
    convection-diffusion system on 128^3 (upwind, velocity (0.5, 0.3, 0.2)
    per grid unit), HBMC order bs = 8, w = 32, FP64, to 1e-8.  A step is one
    hbmc_bicgstab call (inputs resident); the CPU baseline is the oracle's
    BiCGStab on one core over a bounded number of iterations, scaled."""
    import torch
    from paper_1908_00741_gb300 import hbmc as H
    from paper_1908_00741_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    P = W.convection_diffusion_problem(GRID, bs=DEFAULT_BS)
    ctx = H.hbmc_build(P.A, DEFAULT_BS, 32, box=P.box, device=local, nonsymmetric=True)
    stream = torch.cuda.current_stream()
    H.hbmc_set_stream(ctx, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st, bad = H.hbmc_ilu0(ctx)
    e1.record(stream)
    torch.cuda.synchronize()
    assert st == H.OK, bad
    ilu_ms = e0.elapsed_time(e1)
    b = torch.tensor(P.b, device="cuda")
    x = torch.zeros_like(b)
    for _ in range(args.warmup):
        x.zero_()
        res = H.hbmc_bicgstab(ctx, b, x, tol=TOL)
    assert res.status == H.OK, res
    torch.cuda.synchronize()
    barrier(dist)
    with ClockSampler(local) as clk:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        launches = 0
        for _ in range(args.steps):
            x.zero_()
            res = H.hbmc_bicgstab(ctx, b, x, tol=TOL)
            launches += ctx.info()["last_launches"]
        ev[1].record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    ms = max_over_ranks(dist, ev[0].elapsed_time(ev[1]) / args.steps, "cuda")
    err = float(np.max(np.abs(x.cpu().numpy() - P.x_star)) / np.max(np.abs(P.x_star)))
    H.hbmc_set_precision(ctx, H.PREC_F32)
    for _ in range(2):
        x.zero_()
        r32 = H.hbmc_bicgstab(ctx, b, x, tol=TOL)
    a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(5):
        x.zero_()
        r32 = H.hbmc_bicgstab(ctx, b, x, tol=TOL)
    c.record(stream)
    torch.cuda.synchronize()
    f32_ms = a.elapsed_time(c) / 5
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        an = oracle.analyse(P.A, DEFAULT_BS, 32, box=P.box)
        lval, uval, udiag, uinv, _ = oracle.factor_ilu(an)
        k = min(args.cpu_sample_iters, res.iters)
        t = time.perf_counter()
        s = oracle.bicgstab(an, lval, uval, uinv, P.b, tol=TOL, maxit=k)
        dt = time.perf_counter() - t
        cpu = {"value": round(dt / max(s.iters, 1) * res.iters * 1e3, 3), "unit": "ms", "cores": 1,
               "kind": "oracle", "sample": f"{s.iters} BiCGStab iterations of the 128^3 solve ({dt:.2f} s), "
                                           f"scaled to {res.iters} iterations"}
    if rank != 0:
        return
    line = {
        "metric": "ILU(0)-BiCGStab time to 1e-8 FP64 residual (nonsymmetric)", "value": round(ms, 4), "unit": "ms",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"7-point upwind convection-diffusion {GRID}^3 ({P.A.n} unknowns, {P.A.nnz} "
                               f"nonzeros), bs={DEFAULT_BS} (2x2x2 boxes), w=32, tol {TOL:g}",
                   "n": P.A.n, "nnz": P.A.nnz, "bs": DEFAULT_BS, "w": 32, "colors": ctx.info()["nc"]},
        "iters": res.iters, "true_relres": res.true_relres, "max_rel_err_vs_xstar": err,
        "ilu0_ms": round(ilu_ms, 3), "ms_per_iter": round(ms / max(res.iters, 1), 4),
        "f32_substitutions": {"ms": round(f32_ms, 3), "iters": r32.iters, "true_relres": r32.true_relres},
        "gpu_launches": int(launches), "clocks": clk.summary(), "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def run_structural(args):
    """The row-split SpMV (Section 5.2.2's remedy for SELL slices whose rows
    differ much in length) on the Audikw_1-shaped stand-in: 68^3 nodes x 3 DOF
    (943,296 unknowns, about 78M nonzeros, row lengths spread so that SELL
    with slices of 4 / 8 rows processes about 26% / 39% more entries than CRS,
    the paper's 28% / 40% for Audikw_1), natural order, algebraic blocking
    bs = 8, w = 32.  A step is one hbmc_iccg call with the split SpMV
    (pieces of 64 entries, piece cost 2); the same solve without splitting
    and with the variable-slice-height layout (the other remedy, cost 8 per
    sub-slice), the SpMV alone in each layout, and the processed entries are
    reported beside it."""
    import torch
    from paper_1908_00741_gb300 import hbmc as H
    from paper_1908_00741_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    piece = 64
    P = W.structural_problem(args.structural_m)
    A = P.A
    stream = torch.cuda.current_stream()
    ctxs = {}
    loop = H.LOOP_HOST if args.loop == "host" else H.LOOP_GRAPH
    for name, split, vs in (("split", piece, 0), ("plain", 0, 0), ("vslice", 0, 8)):
        c = H.hbmc_build(A, DEFAULT_BS, 32, device=local, sell_split=split, sell_vslice=vs, loop_mode=loop)
        H.hbmc_set_stream(c, stream)
        st, bad = H.hbmc_ic0(c, 0.0)
        assert st == H.OK, bad
        ctxs[name] = c
    ctx = ctxs["split"]
    b = torch.tensor(P.b, device="cuda")
    x = torch.zeros_like(b)

    def solve(c):
        x.zero_()
        return H.hbmc_iccg(c, b, x, tol=TOL)

    for _ in range(args.warmup):
        res = solve(ctx)
    assert res.status == H.OK, res
    torch.cuda.synchronize()
    barrier(dist)
    with ClockSampler(local) as clk:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        launches = 0
        for _ in range(args.steps):
            res = solve(ctx)
            launches += ctx.info()["last_launches"]
        ev[1].record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    ms = max_over_ranks(dist, ev[0].elapsed_time(ev[1]) / args.steps, "cuda")
    err = float(np.max(np.abs(x.cpu().numpy() - P.x_star)) / np.max(np.abs(P.x_star)))

    # the same solve without row splitting, and both with FP32 substitutions
    others = {}
    for name, c, prec in () if args.no_variants else (
            ("plain_f64", ctxs["plain"], H.PREC_F64), ("vslice_f64", ctxs["vslice"], H.PREC_F64),
            ("split_f32", ctx, H.PREC_F32), ("plain_f32", ctxs["plain"], H.PREC_F32)):
        H.hbmc_set_precision(c, prec)
        for _ in range(2):
            r = solve(c)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        a.record(stream)
        for _ in range(reps):
            r = solve(c)
        e.record(stream)
        torch.cuda.synchronize()
        others[name] = {"ms": round(a.elapsed_time(e) / reps, 3), "iters": r.iters, "true_relres": r.true_relres}
        H.hbmc_set_precision(c, H.PREC_F64)

    # e2e through the host-buffer entry point
    bh = torch.tensor(P.b).pin_memory().numpy()
    xh = torch.zeros(A.n, dtype=torch.float64).pin_memory().numpy()
    H.hbmc_iccg_host(ctx, bh, xh, tol=TOL)
    e2e = []
    for _ in range(3):
        xh[:] = 0.0
        t = time.perf_counter()
        H.hbmc_iccg_host(ctx, bh, xh, tol=TOL)
        e2e.append((time.perf_counter() - t) * 1e3)
    e2e_ms = max_over_ranks(dist, statistics.median(e2e), "cuda")

    # one CG iteration's phases in both layouts (CUDA events around back-to-back runs)
    prof = {}
    for name, c in ctxs.items():
        solve(c)
        prof[name] = H.hbmc_profile_kernels(c, 20)
    inf, inf0 = ctx.info(), ctxs["plain"].info()
    peak, peak_kind = measured_peaks()
    sp_bytes = spmv_bytes(A.n, A.nnz)
    sp_fma = A.nnz + A.n
    gbs = {k: sp_bytes / (prof[k]["spmv"] * 1e-3) / 1e9 for k in prof}
    tfl = {k: 2 * sp_fma / (prof[k]["spmv"] * 1e-3) / 1e12 for k in prof}
    roofline = {"bound": "hbm", "kernel": "k_spmv_pieces + k_spmv_split (q = A p, fused p.q)",
                "achieved": round(gbs["split"], 1), "peak": peak, "unit": "GB/s",
                "frac": round(gbs["split"] / peak, 4), "traffic": None, "algorithmic_bytes": sp_bytes,
                "peak_source": peak_kind,
                "fp64": {"fma_per_launch": sp_fma, "achieved_tflops": round(tfl["split"], 4),
                         "peak_tflops": FP64_NOMINAL_TFLOPS, "frac": round(tfl["split"] / FP64_NOMINAL_TFLOPS, 4),
                         "peak_source": "nominal"}}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        an = oracle.analyse(A, DEFAULT_BS, 32)
        lval, _, dinv, _ = oracle.factor(an, 0.0)
        plan = oracle.split_plan(an.row_ptr, 32, piece, 2)
        k = min(args.cpu_sample_iters, res.iters)
        t = time.perf_counter()
        s = oracle.pcg(an, lval, dinv, P.b, tol=TOL, maxit=k, split=plan)
        dt = time.perf_counter() - t
        cpu = {"value": round(dt / max(s.iters, 1) * res.iters * 1e3, 3), "unit": "ms", "cores": 1,
               "kind": "oracle", "sample": f"{s.iters} split-SpMV PCG iterations of the structural solve "
                                           f"({dt:.2f} s), scaled to {res.iters} iterations"}
    if rank != 0:
        return
    line = {
        "metric": "ICCG time to 1e-8 FP64 residual with the row-split SpMV", "value": round(ms, 4), "unit": "ms",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"irregular 3-DOF structural stand-in for Audikw_1, {args.structural_m}^3 nodes "
                               f"({A.n} unknowns, {A.nnz} nonzeros), natural order, algebraic bs={DEFAULT_BS}, "
                               f"w=32, row splitting with pieces of {piece}, tol {TOL:g}",
                   "n": A.n, "nnz": A.nnz, "bs": DEFAULT_BS, "w": 32, "colors": inf["nc"],
                   "l2": f"inputs larger than L2 (device working set {inf['device_bytes'] / 1e9:.2f} GB)"},
        "iters": res.iters, "true_relres": res.true_relres, "max_rel_err_vs_xstar": err,
        "ms_per_iter": round(ms / max(res.iters, 1), 4),
        "processed_entries": {"crs": A.nnz, "sell": inf0["sell_entries_a"], "split": inf["sell_entries_split"],
                              "vslice": ctxs["vslice"].info()["sell_entries_vslice"],
                              "sell_over_crs": round(inf0["sell_entries_a"] / A.nnz, 4),
                              "split_over_crs": round(inf["sell_entries_split"] / A.nnz, 4),
                              "vslice_over_crs": round(ctxs["vslice"].info()["sell_entries_vslice"] / A.nnz, 4),
                              "split_rows": inf["split_rows"], "pieces": inf["split_pieces"]},
        "spmv_ms": {k: round(v["spmv"], 4) for k, v in prof.items()},
        "phase_ms": {k: {q: round(t, 4) for q, t in v.items()} for k, v in prof.items()},
        "spmv_gbs_algorithmic": {k: round(v, 1) for k, v in gbs.items()},
        "variants": others,
        "e2e": {"value": round(e2e_ms, 4), "unit": "ms", "h2d_bytes_per_step": 2 * A.n * 8,
                "d2h_bytes_per_step": A.n * 8},
        "gpu_launches": int(launches), "roofline": roofline, "clocks": clk.summary(), "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def run_reference(args):
    """The reference arm: the CPU oracle as it stands (single-threaded FP64 C)
    on this host's cores, on the GPU arm's workload.  A full solve takes
    seconds per step, so each step is a bounded sample: setup once, then
    `--ref-sample-iters` PCG iterations per step; `value` is the per-iteration
    time scaled to the full solve's iteration count (the GPU solve's, 124 at
    128^3 bs 8), `ms_per_step` the measured time of a sampled step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1908_00741_gb300 import workloads as W

    oracle.build()
    P = W.poisson_problem(GRID, bs=args.bs)
    an = oracle.analyse(P.A, P.bs, P.w, box=P.box)
    lval, _, dinv, _ = oracle.factor(an, 0.0)
    nc = int(an.nc)
    full_iters = args.ref_full_iters
    sample = args.ref_sample_iters

    def step(maxit):
        t = time.perf_counter()
        s = oracle.pcg(an, lval, dinv, P.b, tol=TOL, maxit=maxit)
        dt = time.perf_counter() - t
        return dt, s.iters

    # the start of a solve (r = b - A x0, z = M^-1 r) once, then the sampled steps
    start_s = step(0)[0]
    for _ in range(args.warmup):
        step(sample)
    runs = [step(sample) for _ in range(args.steps)]
    step_s = statistics.mean(dt for dt, _ in runs)
    per_iter = statistics.mean(max(dt - start_s, 0.0) / max(it, 1) for dt, it in runs)
    v = (start_s + per_iter * full_iters) * 1e3
    host = host_info()
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_s * 1e3, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"7-point Poisson {GRID}^3 ({P.A.n} unknowns, {P.A.nnz} nonzeros), "
                               f"bs={args.bs} ({'x'.join(map(str, P.box))} boxes), w=32, FP64 substitutions, "
                               f"tol {TOL:g}",
                   "n": P.A.n, "nnz": P.A.nnz, "bs": args.bs, "w": 32, "colors": nc, "precision": "f64",
                   "loop": "host (single-thread CPU oracle)", "parallelism": "single-thread CPU oracle"},
        "scaled_from_iters": sample, "full_iters": full_iters, "sample_s": round(step_s, 4),
        "cpu_baseline": {"value": round(v, 3), "unit": "ms", "cores": 1, "kind": "oracle",
                         "sample": f"each step: the start of the 128^3 solve and {sample} PCG iterations "
                                   f"({step_s:.3f} s); value = start ({start_s:.3f} s) + per-iteration time "
                                   f"x {full_iters} iterations",
                         "scaled_from_iters": sample, "sample_s": round(step_s, 4), "host": host},
        "e2e": {"value": round(v, 3), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--bs", type=int, default=DEFAULT_BS)
    ap.add_argument("--workload", default="poisson128",
                    choices=["poisson128", "config3", "config5", "batch", "learned", "orderings", "sor", "ilu",
                             "structural"],
                    help="poisson128: the headline solve; config3 / config5: the 27-point 96^3 / 3-DOF 100^3 "
                         "random-order solve (FP32 substitutions unless --precision f64); "
                         "batch: 256 uneven systems solved together; "
                         "learned: learned IC shift against the plain rule; orderings: MC, BMC and HBMC; "
                         "sor: symmetric SOR sweeps; ilu: ILU(0)-BiCGStab on a nonsymmetric system; "
                         "structural: the row-split SpMV on an Audikw_1-shaped matrix")
    ap.add_argument("--sor-sweeps", type=int, default=10)
    ap.add_argument("--learned-train", type=int, default=200)
    ap.add_argument("--learned-heldout", type=int, default=40)
    ap.add_argument("--veclap-m", type=int, default=100)
    ap.add_argument("--structural-m", type=int, default=68)
    ap.add_argument("--hetero-m", type=int, default=96)
    ap.add_argument("--curl-m", type=int, default=70)
    ap.add_argument("--batch-systems", type=int, default=256)
    ap.add_argument("--precision", default=None, choices=["f64", "f32"],
                    help="substitution precision (default: f64 for poisson128, f32 for config3 / config5)")
    ap.add_argument("--loop", default="graph", choices=["graph", "host"],
                    help="graph: one CUDA graph per solve with a device-side while node; "
                         "host: host-driven iterations (kernels visible to ncu)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 27-point, 3-DOF, batch and learned-shift configurations of the default line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-iters", type=int, default=40)
    ap.add_argument("--cpu-config-iters", type=int, default=2,
                    help="PCG iterations of the oracle sampled beside the 27-point and 3-DOF configurations")
    ap.add_argument("--ref-sample-iters", type=int, default=10)
    ap.add_argument("--ref-full-iters", type=int, default=124)
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "f32" if args.workload in ("config3", "config5") else "f64"
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        import __graft_entry__
        __graft_entry__.build()
        {"batch": run_batch, "learned": run_learned, "orderings": run_orderings, "config3": run_config,
         "config5": run_config,
         "sor": run_sor, "ilu": run_ilu, "structural": run_structural}.get(args.workload, run_gpu)(args)


if __name__ == "__main__":
    main()
