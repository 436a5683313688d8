#!/usr/bin/env python3
"""AAR benchmark: solves/s of the 256^3 radius-6 Poisson workload at a 1e-8 FP64 relative residual.

Workload (one step = one complete solve): -lap u = f on a 256^3 interior grid, 12th-order
central-difference Laplacian (radius 6, 37-point star), zero Dirichlet boundary, h = 1,
f = 8 random sine modes + 1e-3 uniform noise (seed 1000), Jacobi AAR with omega = beta = 0.6,
m = 7, p = 6, stopped at ||b - A x|| / ||b|| <= 1e-8 (FP64). The headline form is FP32 inner
AAR solves inside FP64 iterative refinement; the plain FP64 form is timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun each rank solves its own replica (the path has no data-path exchange); rank 0
prints one JSON line. ``--impl reference`` times the CPU oracle (the FP64 reference
implementation written from the paper) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "AAR solves/s + achieved HBM GB/s at 1e-8 FP64 rel. residual; serve p50/p99 ms"
N_SIDE, RADIUS, SEED = 256, 6, 1000
PRM = dict(omega=0.6, beta=0.6, m=7, p=6, tol=1e-8)
WORKLOAD = "poisson3d_r6_256cubed_sines_mixed_fp32_inner_fp64_refinement"
# FP64 AAR iterations of this workload to 1e-8, as counted by the FP64 GPU path (whose iteration
# counts equal the oracle's in the parity tests; a full oracle solve of this size takes about 17
# minutes on one core). It scales the oracle's per-iteration time in the reference arm, which
# runs without a GPU; the CPU-baseline leg uses the count of the same run's FP64 solve.
FP64_ITERS = 815
CONFIG = {
    "workload": WORKLOAD,
    "grid": [N_SIDE, N_SIDE, N_SIDE],
    "radius": RADIUS,
    "rhs": "8 sine modes + 1e-3 uniform noise, seed 1000",
    "omega": PRM["omega"], "beta": PRM["beta"], "m": PRM["m"], "p": PRM["p"], "tol": PRM["tol"],
    "precision": "FP32 inner AAR + FP64 refinement (residual, norm, Gram solve in FP64)",
    "l2": "inputs larger than L2 (history ring + vectors ~1.4 GB per solve)",
}


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(ms_total: float, world: int, device) -> float:
    """The slowest rank's timed span (every rank calls this after its own timed region): replicas
    run the same workload, and the job's time is the time of its last replica."""
    if world <= 1:
        return ms_total
    import torch

    t = torch.tensor([ms_total], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, steps: int, ms_total: float) -> float:
    """Whole-job solves/s: every rank (one replica per GPU) completes `steps` solves in the
    slowest rank's `ms_total`."""
    return world * steps / (ms_total / 1e3)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def alg_bytes_per_solve(n: int, info, m: int, p: int, w: int, mixed: bool) -> float:
    """Algorithmic HBM bytes of one solve, from its iteration counts (one read or write per
    vector touched, halos counted once):
      Richardson sweep 4 words/point; Anderson sweep 3; Gram (c+1);
      update: FP64 literal form 2c+3 (x_k, f_k, c+1 pairs of history columns, x_{k+1}); the mixed
        form's compressed update c+3+2a (c+1 residual columns, x_k, the two x columns of each of
        the a = floor(c/p) window differences made by Anderson steps, x_{k+1});
      mixed only: FP64 residual 8+8+4 bytes, x64 += d 8+4+8 bytes per refinement."""
    iters = info.iterations
    A = info.anderson_steps
    c = m
    upd = (c + 3 + 2 * (c // p)) if mixed else (2 * c + 3)
    per_pt = (iters - A) * 4 * w + A * (3 * w + (c + 1) * w + upd * w)
    if mixed:
        per_pt += (info.refinements + 1) * 20 + info.refinements * 20
    return float(per_pt) * n


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5], parts[6], parts[7], parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def oracle_sample(P, iters: int):
    """Time `iters` FP64 oracle iterations (one Anderson cycle when iters == p) on the host."""
    import oracle

    op = oracle.Operator(P)
    t0 = time.perf_counter()
    r = oracle.solve(P, max_iter=iters, op=op, **dict(PRM, tol=0.0))
    dt = time.perf_counter() - t0
    assert r.iterations == iters
    return dt / iters


def host_cores() -> dict:
    """Cores of the host the oracle runs on: the machine's count and this process's affinity set."""
    try:
        aff = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        aff = None
    return {"nproc": os.cpu_count(), "affinity": aff}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    P = workloads.poisson_sine_modes(N_SIDE, radius=RADIUS, seed=SEED)
    iters_solve = FP64_ITERS
    times = []
    sample_iters = PRM["p"]  # one full Anderson cycle per step (5 Richardson steps, 1 Anderson step)
    for s in range(args.warmup + args.steps):
        t = oracle_sample(P, sample_iters)
        if s >= args.warmup:
            times.append(t)
    s_per_iter = statistics.mean(times)
    value = 1.0 / (s_per_iter * iters_solve) if iters_solve else None
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": s_per_iter * sample_iters * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": CONFIG,  # the same workload and stopping rule as the GPU arm
        "impl": "reference", "reference_form": f"plain FP64 AAR (the oracle), {iters_solve} iterations per solve",
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "host": host_cores(), "kind": "oracle",
                         "sample": f"one Anderson cycle ({sample_iters} FP64 oracle iterations) on the full grid "
                                   f"per step, scaled by the {iters_solve} iterations a full FP64 solve takes "
                                   f"(the FP64 GPU path's count of this workload; its counts equal the oracle's "
                                   f"in the parity tests)"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "s_per_iteration": s_per_iter,
    }
    print(json.dumps(line))
    return 0


def kernel_traffic(kernel_src_hash: str):
    """(read + write, read, write) DRAM bytes per launch of the FP32 sweep from the committed ncu
    summary, or Nones when the kernel source changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "sweep_fp32_r6_256.md")
    if not os.path.exists(p):
        return None, None, None
    text = open(p).read()
    mh = re.search(r"kernel source sha256:\s*([0-9a-f]+)", text)
    if not mh or mh.group(1) != kernel_src_hash:
        return None, None, None
    vals = []
    for key in ("traffic_bytes_per_launch", "dram_read_bytes_per_launch", "dram_write_bytes_per_launch"):
        m = re.search(key + r":\s*([0-9.eE+]+)", text)
        vals.append(float(m.group(1)) if m else None)
    return tuple(vals)


def stencil_src_hash() -> str:
    h = hashlib.sha256()
    for f in ["aar_stencil_tma.cuh", "aar_stencil.cuh", "aar_engine.cuh", "aar_mbar.cuh", "aar_fp64.cuh"]:
        h.update(open(os.path.join(ROOT, "paper_1606_08740_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def run_small_case():
    """Profiling run for ncu (no JSON line): two FP64 solves of the 32^3 7-point Poisson workload
    to 1e-8 (with AAR_HOST_LOOP=1 every kernel of the solve is a separate launch)."""
    import torch

    from paper_1606_08740_gb300 import aar

    P = workloads.poisson_uniform(32, radius=1, seed=0)
    b = torch.from_numpy(P.b).cuda()
    x = torch.empty_like(b)
    with aar.Solver.stencil(aar.desc_of(P), aar.FP64) as s:
        for _ in range(2):
            r = s.solve(b, x, prm=aar.params(omega=0.6, beta=0.6, m=7, p=6, tol=1e-8))
        print("solve", r)
    return 0


def run_batch_case():
    """Profiling run for ncu (no JSON line): one batched mixed solve of the 512 Helmholtz systems
    (tiles from the autotuner), after a warm-up batch solve."""
    import torch

    from paper_1606_08740_gb300 import aar, autotune

    probs = workloads.batched_helmholtz(512, seed_base=3000)
    descs = [aar.desc_of(P) for P in probs]
    autotune.tune(descs, aar.MIXED, 7)
    bs = [torch.from_numpy(P.b).cuda() for P in probs]
    xs = [torch.empty_like(b) for b in bs]
    bt = aar.Batch(descs, aar.MIXED)
    for _ in range(2):
        res = bt.solve(bs, xs, aar.params(omega=0.6, beta=0.6, m=7, p=6, tol=1e-8))
    bt.close()
    print("batch", max(r.iterations for r in res), sum(r.iterations for r in res) / len(res), res[0].launches)
    return 0


def run_csr_case():
    """Profiling run for ncu (no JSON line): the 128^3 upwind CSR workload in FP64, a 12-iteration
    solve, then the CSR sweep launched 3 times through aar_profile_kernel."""
    import torch

    from paper_1606_08740_gb300 import aar

    P = workloads.convection_diffusion(128, seed=2000)
    rp, ci, va = (torch.from_numpy(a).cuda() for a in (P.row_ptr, P.col_idx, P.val))
    b = torch.from_numpy(P.b).cuda()
    x = torch.empty_like(b)
    with aar.Solver.csr(rp, ci, va, aar.FP64) as s:
        r = s.solve(b, x, prm=aar.params(omega=0.5, beta=0.5, m=10, p=5, tol=0.0, max_iter=12), raise_on_error=False)
        print("setup", r)
        print(aar.K_SWEEP, s.profile_kernel(aar.K_SWEEP, 3))
    return 0


def run_profile_case(args):
    """Small, fixed launch sequences for ncu (no JSON line)."""
    import torch

    from paper_1606_08740_gb300 import aar

    P = workloads.poisson_sine_modes(N_SIDE, radius=RADIUS, seed=SEED)
    b = torch.from_numpy(P.b).cuda()
    x = torch.empty_like(b)
    d = aar.desc_of(P)
    d.block = 2 if args.block else 0
    with aar.Solver.stencil(d, aar.MIXED) as s:
        if args.profile_solve:
            for _ in range(2):
                r = s.solve(b, x, prm=aar.params(**PRM))
            print("solve", r)
        else:
            r = s.solve(b, x, prm=aar.params(**dict(PRM, max_iter=14)), raise_on_error=False)
            print("setup", r)
            for k in [aar.K_SWEEP, aar.K_SWEEP_ANDERSON, aar.K_GRAM, aar.K_UPDATE, aar.K_RESID64, aar.K_FINALIZE]:
                print(k, s.profile_kernel(k, 3))
    return 0


def run_periodic(aar, torch, dev, stream, n: int = 256):
    """Periodic boundaries with the paper's sixth-order stencil (radius 3, Sec. 3.2/3.3): n^3
    Poisson, f = 8 random Fourier modes + 1e-3 noise, zero mean (seed 5000); mixed and plain FP64
    solves to 1e-8, the FP32 sweep's algorithmic bandwidth, and the mixed solution's error against
    the FP64 one (both zero-mean: periodic Poisson determines u up to a constant)."""
    P = workloads.periodic_modes(n, radius=3, seed=5000)
    b = torch.from_numpy(P.b).to(dev)
    x = torch.empty_like(b)
    prm = aar.params(**PRM)
    desc = aar.desc_of(P)
    out = {"workload": f"poisson3d_r3_{n}cubed_periodic_fourier_modes", "grid": [n, n, n], "radius": 3}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        with aar.Solver.stencil(desc, aar.MIXED, stream=stream) as s:
            r = s.solve(b, x, prm=prm)
            torch.cuda.synchronize()
            e0.record(stream)
            r = s.solve(b, x, prm=prm)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            sweep_ms = s.profile_kernel(aar.K_SWEEP, 10)
            out.update(mixed_solves_per_s=1e3 / ms, mixed_ms=ms, mixed_iterations=r.iterations,
                       mixed_refinements=r.refinements, mixed_status=r.status, rel_residual_fp64=s.rel_residual(b, x),
                       sweep_fp32_ms=sweep_ms, sweep_fp32_gbs=16.0 * P.n / (sweep_ms * 1e-3) / 1e9)
        x_mixed = x.clone()
        with aar.Solver.stencil(desc, aar.FP64, stream=stream) as s:
            e0.record(stream)
            r = s.solve(b, x, prm=prm)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            out.update(fp64_solves_per_s=1e3 / ms, fp64_ms=ms, fp64_iterations=r.iterations, fp64_status=r.status)
        dm, d64 = x_mixed - x_mixed.mean(), x - x.mean()
        out["mixed_error_vs_gpu_fp64"] = float(torch.linalg.vector_norm(dm - d64) / torch.linalg.vector_norm(d64))
    del x, b
    return out


def run_block(aar, torch, dev, stream, jacobi_ms: float | None, periodic_jacobi_ms: float | None):
    """Block Jacobi with 2 x 2 x 2 boxes (row f4: the block Jacobi of Sec. 3.2/3.3 with exact block
    solves, fused into the paired FP32 sweep): the headline workload (256^3 radius-6 Poisson, sine
    modes, tol 1e-8) in the mixed and plain FP64 forms, and the 256^3 periodic sixth-order case
    in the mixed form; Jacobi figures of the same run beside them."""
    out = {}
    cases = [("poisson3d_r6_256cubed_sines", workloads.poisson_sine_modes(N_SIDE, radius=RADIUS, seed=SEED),
              jacobi_ms, True),
             ("poisson3d_r3_256cubed_periodic_fourier_modes", workloads.periodic_modes(256, radius=3, seed=5000),
              periodic_jacobi_ms, False)]
    prm = aar.params(**PRM)
    for name, P, jms, with_fp64 in cases:
        b = torch.from_numpy(P.b).to(dev)
        x = torch.empty_like(b)
        d = aar.desc_of(P)
        d.block = 2
        e = {"workload": name, "block": [2, 2, 2]}
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for key, prec in (("mixed", aar.MIXED), ("fp64", aar.FP64)):
                if key == "fp64" and not with_fp64:
                    continue
                with aar.Solver.stencil(d, prec, stream=stream) as s:
                    r = s.solve(b, x, prm=prm)
                    torch.cuda.synchronize()
                    e0.record(stream)
                    r = s.solve(b, x, prm=prm)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1)
                    entry = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "iterations": r.iterations,
                             "refinements": r.refinements, "status": r.status,
                             "rel_residual_fp64": s.rel_residual(b, x)}
                    if prec == aar.MIXED:
                        t = s.profile_kernel(aar.K_SWEEP, 20)
                        peak, kind = load_peaks()
                        gbs = 16.0 * P.n / (t * 1e-3) / 1e9
                        entry["sweep_ms"] = t
                        entry["sweep_roofline"] = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                                   "frac": gbs / peak, "peak_kind": kind}
                e[key] = entry
        if jms:
            e["mixed_speedup_vs_jacobi"] = jms / e["mixed"]["ms_per_solve"]
        out[name] = e
        del b, x
    return out


def measure_fp64_peak(aar, stream, local: int):
    """Measured FP64 instruction rates (thread-level instructions/s) of DFMA and DADD chains that
    fill every SM (aar_measure_fp64_rate), best of three each, with the SM clock sampled while
    they run: the denominator of the FP64 sweeps' ALU roofline."""
    with ClockSampler(local) as clk:
        dfma = max(aar.measure_fp64_rate(0, stream) for _ in range(3))
        dadd = max(aar.measure_fp64_rate(1, stream) for _ in range(3))
    return {"dfma_per_s": dfma, "dadd_per_s": dadd, "clocks": clk.summary(),
            "how": "aar_measure_fp64_rate: 8 independent chains per thread, grid filling every SM, CUDA events"}


def fp64_mix_peak(fp64: dict | None, n_add: int, n_fma: int) -> tuple[float, str]:
    """FP64 instruction peak of a kernel running n_add DADD and n_fma DFMA/DMUL instructions per
    point: the rate at which the measured pipes retire that mix; the nominal 1.25 TFLOP/s FP64
    (0.625e12 DFMA/s) when nothing was measured."""
    if not fp64:
        return 1.25e12 / 2, "nominal"
    t = n_add / fp64["dadd_per_s"] + n_fma / fp64["dfma_per_s"]
    return (n_add + n_fma) / t, "measured"


def run_small_poisson(aar, torch, dev, stream, cpu: bool, steps: int = 20):
    """The small oracle-sized workload: 32^3 7-point Poisson, h = 1, zero Dirichlet, f uniform
    [-1, 1] (seed 0), plain FP64 Jacobi AAR, omega = beta = 0.6, m = 7, p = 6, tol 1e-8 (its working
    set, about 5 MB, stays in L2: latency-bound, so solves/s and us per iteration, no HBM
    roofline). With cpu: one full oracle solve of the same system timed on the host, with the
    oracle's own iteration count."""
    P = workloads.poisson_uniform(32, radius=1, seed=0)
    b = torch.from_numpy(P.b).to(dev)
    x = torch.empty_like(b)
    prm = aar.params(omega=0.6, beta=0.6, m=7, p=6, tol=1e-8)
    out = {"workload": "poisson3d_7pt_32cubed_uniform_fp64", "grid": [32, 32, 32], "radius": 1, "tol": 1e-8}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        with aar.Solver.stencil(aar.desc_of(P), aar.FP64, stream=stream) as s:
            for _ in range(3):
                r = s.solve(b, x, prm=prm)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(steps):
                r = s.solve(b, x, prm=prm)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            out.update(solves_per_s=1e3 / ms, ms_per_solve=ms, iterations=r.iterations,
                       anderson_steps=r.anderson_steps, us_per_iteration=1e3 * ms / max(1, r.iterations),
                       status=r.status, rel_residual_fp64=s.rel_residual(b, x), launches_per_solve=r.launches)
    if cpu:
        import oracle

        t0 = time.perf_counter()
        ro = oracle.solve(P, omega=0.6, beta=0.6, m=7, p=6, tol=1e-8)
        dt = time.perf_counter() - t0
        out["cpu_oracle"] = {"value": 1.0 / dt, "unit": "solves/s", "seconds": dt, "cores": 1, "host": host_cores(),
                             "kind": "oracle", "iterations": ro.iterations,
                             "sample": "one full FP64 oracle solve of this system (its own iteration count)"}
        out["iterations_match_oracle"] = ro.iterations == out["iterations"]
    del b, x
    return out


def run_csr(aar, torch, dev, stream, fp64: dict | None, steps: int = 1):
    """The nonsymmetric sparse workload: 128^3 first-order upwind convection-diffusion in CSR
    (int32 indices, FP64 values; velocity of 16 Fourier modes at cell Peclet 5, seed 2000), f
    uniform, Jacobi AAR with omega = beta = 0.5, m = 10, p = 5, tol 1e-8, in the plain FP64 form
    (about 21k iterations), with the CSR sweep's roofline. The mixed form is left out: its FP32
    inner solves stall on this system long before the 1e-8 target (30 refinements ended at a
    relative residual of 4.6e-3 when it was tried)."""
    P = workloads.convection_diffusion(128, seed=2000)
    n, nnz = P.n, int(P.row_ptr[-1])
    rp = torch.from_numpy(P.row_ptr).to(dev)
    ci = torch.from_numpy(P.col_idx).to(dev)
    va = torch.from_numpy(P.val).to(dev)
    b = torch.from_numpy(P.b).to(dev)
    x = torch.empty_like(b)
    prm = aar.params(omega=0.5, beta=0.5, m=10, p=5, tol=1e-8)
    out = {"workload": "convection_diffusion_upwind_128cubed_csr", "rows": n, "nnz": nnz, "tol": 1e-8,
           "m": 10, "p": 5, "omega": 0.5, "beta": 0.5}
    peak, kind = load_peaks()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, prec in (("fp64", aar.FP64),):
        with torch.cuda.stream(stream):
            with aar.Solver.csr(rp, ci, va, prec, stream=stream) as s:
                # warm-up: the solve graph and tables, on a short solve
                s.solve(b, x, prm=aar.params(omega=0.5, beta=0.5, m=10, p=5, tol=1e-8, max_iter=50),
                        raise_on_error=False)
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(steps):
                    r = s.solve(b, x, prm=prm)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / steps
                t = s.profile_kernel(aar.K_SWEEP, 20)
                # one Richardson sweep: col_idx + val per nonzero; row_ptr, M^{-1}, x_k (gathered
                # from L2 after its first read), b read and f_k, x_{k+1} written per row
                if prec == aar.FP64:
                    alg = 12.0 * nnz + (4 + 8 + 8 + 8 + 8 + 8) * n
                else:
                    alg = 8.0 * nnz + (4 + 4 + 4 + 4 + 4 + 4) * n
                gbs = alg / (t * 1e-3) / 1e9
                e = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "iterations": r.iterations,
                     "anderson_steps": r.anderson_steps, "refinements": r.refinements, "status": r.status,
                     "eigen_steps": r.eigen_steps, "rel_residual_fp64": s.rel_residual(b, x), "sweep_ms": t,
                     "sweep_roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                        "frac": gbs / peak, "peak_kind": kind, "alg_bytes_per_launch": alg,
                                        "kernel": f"k_csr<{'double' if prec == aar.FP64 else 'float'}, sweep>"}}
        out[name] = e
    del rp, ci, va, b, x
    return out


def run_complex_case(kind: str):
    """Small, fixed launch sequences of the complex solver for ncu (no JSON line). kind:
    'mixed' / 'fp64': the Eq. 7 cell of 12 x 12 x 12 aluminium cells (192^3, inputs larger than
    L2), a 14-iteration solve, then each solve-loop kernel launched 3 times through
    aar_zprofile_kernel; 'mixed-solve': one complete mixed solve of the 256^3 cell to 1e-6."""
    import torch

    from paper_1606_08740_gb300 import aar

    cells = 16 if kind == "mixed-solve" else 12
    P = workloads.ofdft_helmholtz(cells, 0.486, seed=6000)
    b = torch.from_numpy(P.b).cuda()
    x = torch.empty_like(b)
    prec = aar.FP64 if kind == "fp64" else aar.MIXED
    with aar.ZSolver(aar.zdesc_of(P), prec) as s:
        if kind == "mixed-solve":
            print("solve", s.solve(b, x, prm=aar.zparams(tol=1e-6)))
            return 0
        r = s.solve(b, x, prm=aar.zparams(tol=1e-6, max_iter=14), raise_on_error=False)
        print("setup", r)
        ks = [aar.K_SWEEP, aar.K_SWEEP_ANDERSON, aar.K_GRAM, aar.K_UPDATE, aar.K_FINALIZE]
        if prec == aar.MIXED:
            ks.append(aar.K_RESID64)
        for k in ks:
            print(k, s.profile_kernel(k, 3))
    return 0


def run_complex(aar, torch, dev, stream, cpu: bool = True, fp64: dict | None = None):
    """Complex-valued AAR (Sec. 2 over C) on the OF-DFT kernel-potential equation of Eq. 7:
    -(1/(4 pi)) lap V + Q V = P rho^alpha, sixth-order stencil, periodic, Jacobi, x0 = 0, tol 1e-6
    (Sec. 3.2), rho a stand-in density of displaced FCC aluminium atoms (seed 6000). Two cells at
    the paper's mesh h = 0.486 Bohr: the 3 x 3 x 3 supercell of Sec. 3.2 (48^3) and a 16 x 16 x 16
    one (256^3, the weak-scaling direction of Fig. 4b). Both forms: plain FP64 and the mixed form
    (FP32 inner solves in FP64 refinement), with per-kernel times, the FP64 sweep's FP64 issue rate
    (its bound on this part: FP64 at 1/64 of the FP32 rate) and the FP32 sweep's algorithmic HBM
    bandwidth."""
    out = {}
    prm = aar.zparams(tol=1e-6)
    for cells in (3, 16):
        P = workloads.ofdft_helmholtz(cells, 0.486, seed=6000)
        n = P.n
        b = torch.from_numpy(P.b).to(dev)
        x = torch.empty_like(b)
        entry = {"workload": f"ofdft_helmholtz_al{cells}x{cells}x{cells}_h0.486_{P.nx}cubed", "grid": [P.nx] * 3,
                 "radius": 3, "tol": 1e-6}
        sols = {}
        for name, prec in (("fp64", aar.FP64), ("mixed", aar.MIXED)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                with aar.ZSolver(aar.zdesc_of(P), prec, stream=stream) as s:
                    r = s.solve(b, x, prm=prm)
                    torch.cuda.synchronize()
                    reps = 3 if cells == 3 else 1
                    e0.record(stream)
                    for _ in range(reps):
                        r = s.solve(b, x, prm=prm)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / reps
                    rr = s.rel_residual(b, x)
                    names = ["K_SWEEP", "K_SWEEP_ANDERSON", "K_GRAM", "K_UPDATE", "K_FINALIZE"]
                    if prec == aar.MIXED:
                        names.append("K_RESID64")
                    kt = {k: s.profile_kernel(getattr(aar, k), 10) for k in names}
            sols[name] = x.clone()
            e = {"dtype": "c128" if prec == aar.FP64 else "c64+c128", "solves_per_s": 1e3 / ms, "ms_per_solve": ms,
                 "iterations": r.iterations, "anderson_steps": r.anderson_steps, "refinements": r.refinements,
                 "status": r.status, "rel_residual_fp64": rr, "eigen_steps": r.eigen_steps, "kernel_ms": kt}
            if cells == 16:
                t = kt["K_SWEEP"] * 1e-3
                if prec == aar.FP64:
                    # FP64 instructions per point of the radius-3 complex Richardson sweep: per
                    # component 5 sums per ring (6 neighbours, issued as multiply-adds with a unit
                    # multiplier) and one multiply-add by the real weight, then the centre
                    # coefficient, M^{-1} and omega as multiply-adds; the residual's two adds
                    n_add, n_fma = 2, 2 * 5 * 3 + 2 * 3 + 12
                    dp_instr = n_add + n_fma  # 14 r + 14 at r = 3
                    dp_peak, pk = fp64_mix_peak(fp64, n_add, n_fma)
                    e["sweep_roofline"] = {"bound": "alu", "achieved": dp_instr * n / t / 1e12,
                                           "peak": dp_peak / 1e12, "unit": "TDPinstr/s", "peak_kind": pk,
                                           "frac": dp_instr * n / t / dp_peak, "hbm_gbs": 64.0 * n / t / 1e9}
                else:
                    peak, kind = load_peaks()
                    gbs = 32.0 * n / t / 1e9  # x, b read, f, x_{k+1} written: 4 complex FP32 words per point
                    e["sweep_roofline"] = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                           "frac": gbs / peak, "peak_kind": kind}
            entry[name] = e
        d = sols["mixed"] - sols["fp64"]
        entry["mixed_error_vs_gpu_fp64"] = float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(sols["fp64"]))
        entry["mixed_over_fp64"] = entry["fp64"]["ms_per_solve"] / entry["mixed"]["ms_per_solve"]
        if cells == 3 and cpu:
            import oracle

            t0 = time.perf_counter()
            ro = oracle.zsolve(P, tol=1e-6)
            dt = time.perf_counter() - t0
            entry["cpu_oracle"] = {"value": 1.0 / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                   "iterations": ro.iterations, "sample": "one full FP64 oracle solve of this cell"}
        out[f"al{cells}"] = entry
        del b, x, sols
    return out


def run_complex_block(aar, torch, dev, stream, jacobi: dict | None):
    """Eq. 7 with block Jacobi on 2 x 2 x 2 boxes (the block-Jacobi Helmholtz runs of Sec. 3.2,
    exact block solves): the same two cells as run_complex, plain FP64 and mixed, tol 1e-6, with
    the Jacobi figures of the same run beside them."""
    out = {}
    prm = aar.zparams(tol=1e-6)
    for cells in (3, 16):
        P = workloads.ofdft_helmholtz(cells, 0.486, seed=6000)
        b = torch.from_numpy(P.b).to(dev)
        x = torch.empty_like(b)
        entry = {"workload": f"ofdft_helmholtz_al{cells}x{cells}x{cells}_h0.486_{P.nx}cubed", "block": [2, 2, 2]}
        for name, prec in (("fp64", aar.FP64), ("mixed", aar.MIXED)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                with aar.ZSolver(aar.zdesc_of(P, block=2), prec, stream=stream) as s:
                    r = s.solve(b, x, prm=prm)
                    torch.cuda.synchronize()
                    reps = 3 if cells == 3 else 1
                    e0.record(stream)
                    for _ in range(reps):
                        r = s.solve(b, x, prm=prm)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / reps
                    e = {"solves_per_s": 1e3 / ms, "ms_per_solve": ms, "iterations": r.iterations,
                         "refinements": r.refinements, "status": r.status, "rel_residual_fp64": s.rel_residual(b, x),
                         "block_ms": s.profile_kernel(aar.K_BLOCK, 10), "sweep_ms": s.profile_kernel(aar.K_SWEEP, 10)}
            if jacobi and f"al{cells}" in jacobi:
                e["speedup_vs_jacobi"] = jacobi[f"al{cells}"][name]["ms_per_solve"] / ms
                e["jacobi_iterations"] = jacobi[f"al{cells}"][name]["iterations"]
            entry[name] = e
        out[f"al{cells}"] = entry
        del b, x
    return out


def run_batched(aar, torch, dev, stream, steps: int = 2):
    """512 independent Helmholtz systems (-lap + c) u = f, 7-point, sides log-uniform in [16, 96],
    c in [0.1, 2], f uniform (seeds 3000 + i): one batch per step, FP32 inner + FP64 refinement,
    tiles from the autotuner; the plain FP64 batch is timed beside it."""
    from paper_1606_08740_gb300 import autotune

    probs = workloads.batched_helmholtz(512, seed_base=3000)
    descs = [aar.desc_of(P) for P in probs]
    t0 = time.perf_counter()
    chosen = autotune.tune(descs, aar.MIXED, 7, stream=stream)
    tune_s = time.perf_counter() - t0
    bs = [torch.from_numpy(P.b).to(dev) for P in probs]
    xs = [torch.empty_like(b) for b in bs]
    prm = aar.params(omega=0.6, beta=0.6, m=7, p=6, tol=1e-8)
    out = {"systems": len(probs), "unknowns": int(sum(P.n for P in probs)), "tune_s": tune_s,
           "tile_choices": len(chosen)}
    with torch.cuda.stream(stream):
        bt = aar.Batch(descs, aar.MIXED, stream=stream)
        bt.solve(bs, xs, prm)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            res = bt.solve(bs, xs, prm)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        bt.close()
        out.update(solves_per_s=len(probs) / (ms * 1e-3), ms_per_batch=ms,
                   all_converged=all(r.status == aar.OK for r in res),
                   iterations_max=max(r.iterations for r in res),
                   iterations_mean=sum(r.iterations for r in res) / len(res),
                   refinements_max=max(r.refinements for r in res))
        # FP64 true residuals of a sample, by the library's own FP64 residual check
        worst = 0.0
        for i in range(0, len(probs), 64):
            with aar.Solver.stencil(descs[i], aar.FP64, stream=stream) as s1:
                worst = max(worst, s1.rel_residual(bs[i], xs[i]))
        out["max_rel_residual_sampled"] = worst
        b64 = aar.Batch([aar.desc_of(P) for P in probs], aar.FP64, stream=stream)
        b64.solve(bs, xs, prm)
        torch.cuda.synchronize()
        e0.record(stream)
        b64.solve(bs, xs, prm)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        b64.close()
        out.update(fp64_solves_per_s=len(probs) / (ms64 * 1e-3), fp64_ms_per_batch=ms64,
                   mixed_over_fp64=ms64 / ms)
    del xs, bs
    return out


SERVE_SIDES = (32, 48, 64, 96, 128, 192)


def serve_stream(aar, torch, stream, reqs, descs, pool, budget, ticks=12):
    """Replay a request stream against one server in real time (open loop): each request is
    submitted once its arrival time has passed; latency = completion seen - scheduled arrival.
    Each scheduling round runs 12 ticks (two bodies of the p = 6 tick layout): shorter rounds
    spend more time retiring and admitting (6 ticks: about 93 solves/s of capacity, 12: 100)."""
    sv = aar.Server(6, aar.MIXED, budget_bytes=budget, max_active=1024, stream=stream)
    bufs = {s: [] for s in SERVE_SIDES}
    meta, lat, status = {}, [], []
    t0 = time.perf_counter()
    i = 0
    while i < len(reqs) or meta:
        now = time.perf_counter() - t0
        while i < len(reqs) and reqs[i].arrival_s <= now:
            r = reqs[i]
            x = bufs[r.side].pop() if bufs[r.side] else torch.empty(r.side ** 3, dtype=torch.float64).pin_memory().numpy()
            d = aar.StencilDesc.from_buffer_copy(descs[r.side])
            d.shift = r.shift
            rid = sv.submit(d, pool[r.side][r.rid % len(pool[r.side])], x, aar.params(tol=r.tol, **SERVE_PRM))
            meta[rid] = (r.arrival_s, r.side, x)
            i += 1
        if meta:
            sv.run(ticks)
        elif i < len(reqs):
            time.sleep(max(0.0, min(0.01, reqs[i].arrival_s - now)))
        for rid, res in sv.poll():
            arr, side, x = meta.pop(rid)
            lat.append(time.perf_counter() - t0 - arr)
            status.append(res.status)
            bufs[side].append(x)
    elapsed = time.perf_counter() - t0
    sv.close()
    lat_ms = sorted(1e3 * v for v in lat)
    q = lambda f: lat_ms[min(len(lat_ms) - 1, int(f * len(lat_ms)))] if lat_ms else None  # noqa: E731
    return {"requests": len(reqs), "p50_ms": q(0.50), "p99_ms": q(0.99), "solves_per_s": len(reqs) / elapsed,
            "wall_s": elapsed, "all_converged": all(s_ == aar.OK for s_ in status)}


SERVE_PRM = dict(omega=0.6, beta=0.6, m=7, p=6)


def run_serving(aar, torch, stream, sustain_s=6.0, literal_s=0.3):
    """Continuous-batching serving of radius-6 Poisson/Helmholtz solves, sides uniform over
    {32, 48, 64, 96, 128, 192}, tolerance uniform over {1e-6, 1e-8, 1e-10}, 50/50 Poisson/Helmholtz
    (c uniform in [0.1, 2]), FP32 inner + FP64 refinement, m = 7, p = 6, omega = beta = 0.6.
    Right-hand sides come from a seeded pool of two per side. After an untimed warm-up burst, three
    runs: a closed burst measures capacity; an open-loop Poisson stream at 70% of it gives the
    sustained latency; the literal 2000 req/s stream runs for a short window and drains."""
    from paper_1606_08740_gb300 import autotune

    pool = {s: [workloads.uniform_rhs(s ** 3, 4000 * 1000 + 10 * s + j) for j in range(2)] for s in SERVE_SIDES}
    descs = {s: aar.desc_of(workloads.poisson_uniform(s, radius=6, seed=0)) for s in SERVE_SIDES}
    autotune.tune(list(descs.values()), aar.MIXED, 7, stream=stream)
    budget = 64 << 30
    # warm-up: a closed burst of the capacity burst's size (first allocations of the server's
    # memory pool, first tile lists and tensor maps), not timed
    warm = workloads.serving_requests(2000.0, 10.0, seed=4002, max_requests=96)
    for r in warm:
        r.arrival_s = 0.0
    serve_stream(aar, torch, stream, warm, descs, pool, budget)
    burst = workloads.serving_requests(2000.0, 10.0, seed=4000, max_requests=96)
    for r in burst:
        r.arrival_s = 0.0
    cap = serve_stream(aar, torch, stream, burst, descs, pool, budget)
    rate = 0.7 * cap["solves_per_s"]
    sustained = serve_stream(aar, torch, stream, workloads.serving_requests(rate, sustain_s, seed=4001), descs, pool,
                             budget)
    sustained["offered_req_per_s"] = rate
    literal = serve_stream(aar, torch, stream, workloads.serving_requests(2000.0, literal_s, seed=4000), descs, pool,
                           budget)
    literal["offered_req_per_s"] = 2000.0
    literal["window_s"] = literal_s
    return {"capacity_solves_per_s": cap["solves_per_s"], "burst": cap, "sustained_70pct": sustained,
            "literal_2000_per_s": literal, "p50_ms": sustained["p50_ms"], "p99_ms": sustained["p99_ms"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--plain-steps", type=int, default=1, help="timed plain FP64 solves (0 = skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-system batched measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-periodic", action="store_true", help="skip the periodic-boundary measurement")
    ap.add_argument("--no-complex", action="store_true", help="skip the complex-valued (Eq. 7) measurement")
    ap.add_argument("--no-block", action="store_true", help="skip the block-Jacobi measurement")
    ap.add_argument("--no-small", action="store_true", help="skip the 32^3 7-point FP64 measurement")
    ap.add_argument("--no-csr", action="store_true", help="skip the 128^3 CSR measurement")
    ap.add_argument("--serve-only", action="store_true", help="print only the serving measurement")
    ap.add_argument("--profile-solve", action="store_true",
                    help="profiling run for ncu: one warm-up and one timed mixed solve, nothing else")
    ap.add_argument("--kernel-case", action="store_true",
                    help="profiling run for ncu: a 14-iteration mixed solve, then each solve-loop kernel "
                         "launched 3 times through aar_profile_kernel")
    ap.add_argument("--block", action="store_true",
                    help="with --kernel-case / --profile-solve: block Jacobi (2 x 2 x 2 boxes) in place of Jacobi")
    ap.add_argument("--complex-case", choices=["mixed", "fp64", "mixed-solve"],
                    help="profiling run for ncu of the complex solver (see run_complex_case)")
    ap.add_argument("--small-case", action="store_true",
                    help="profiling run for ncu: two FP64 solves of the 32^3 7-point workload")
    ap.add_argument("--batch-case", action="store_true",
                    help="profiling run for ncu: two batched mixed solves of the 512 Helmholtz systems")
    ap.add_argument("--csr-case", action="store_true",
                    help="profiling run for ncu: the 128^3 CSR workload, 12 FP64 iterations, 3 sweeps")
    args = ap.parse_args()
    if args.small_case:
        return run_small_case()
    if args.csr_case:
        return run_csr_case()
    if args.batch_case:
        return run_batch_case()
    if args.complex_case:
        return run_complex_case(args.complex_case)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_solve or args.kernel_case:
        return run_profile_case(args)
    if args.serve_only:
        import torch

        from paper_1606_08740_gb300 import aar

        print(json.dumps(run_serving(aar, torch, torch.cuda.Stream())))
        return 0

    import torch

    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1606_08740_gb300 import aar

    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    P = workloads.poisson_sine_modes(N_SIDE, radius=RADIUS, seed=SEED)
    n = P.n
    b = torch.from_numpy(P.b).to(dev)
    x = torch.empty_like(b)
    prm = aar.params(**PRM)
    desc = aar.desc_of(P)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # ---- headline: mixed precision, device-resident inputs
    mixed = aar.Solver.stencil(desc, aar.MIXED, stream=stream)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            res = mixed.solve(b, x, prm=prm)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        launches = 0
        infos = []
        with ClockSampler(local) as clk:
            torch.cuda.synchronize()
            barrier()
            e0.record(stream)
            for _ in range(args.steps):
                res = mixed.solve(b, x, prm=prm)
                infos.append(res)
                launches += res.launches
            e1.record(stream)
            torch.cuda.synchronize()
        barrier()
    ms_total = max_over_ranks(e0.elapsed_time(e1), world, dev)
    ms_step = ms_total / args.steps
    value = job_rate(world, args.steps, ms_total)
    ok = all(r.status == aar.OK for r in infos)
    r_true = mixed.rel_residual(b, x)
    info = infos[-1]
    hbm_bytes = alg_bytes_per_solve(n, info, PRM["m"], PRM["p"], 4, True)

    # ---- dominant kernel: the FP32 radius-6 Richardson sweep, timed live on the same stream
    peak, peak_kind = load_peaks()
    sweep_ms = mixed.profile_kernel(aar.K_SWEEP, 20)
    kernel_times = {
        "sweep_fp32": sweep_ms,
        "sweep_anderson_fp32": mixed.profile_kernel(aar.K_SWEEP_ANDERSON, 5),
        "gram_fp32": mixed.profile_kernel(aar.K_GRAM, 5),
        "update_fp32": mixed.profile_kernel(aar.K_UPDATE, 5),
        "resid_fp64": mixed.profile_kernel(aar.K_RESID64, 3),
    }
    sweep_bytes = 16.0 * n  # read x_k, b; write f_k, x_{k+1} (FP32)
    achieved = sweep_bytes / (sweep_ms * 1e-3) / 1e9
    traffic, traffic_rd, traffic_wr = kernel_traffic(stencil_src_hash())
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_read": traffic_rd, "traffic_write": traffic_wr, "kernel": "k_sweep_tma2<6,2,3,2,2> (FP32 radius-6 Richardson sweep)",
                "alg_bytes_per_launch": sweep_bytes, "ms_per_launch": sweep_ms, "peak_kind": peak_kind}

    # ---- end to end through the C ABI with pinned host buffers (copies inside the timed region)
    bh = torch.from_numpy(P.b).pin_memory()
    xh = torch.empty(n, dtype=torch.float64).pin_memory()
    bh_np, xh_np = bh.numpy(), xh.numpy()
    e2e_steps = max(1, min(args.steps, 3))
    mixed.solve(bh_np, xh_np, prm=prm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        mixed.solve(bh_np, xh_np, prm=prm)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": world / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n}
    mixed.close()

    # ---- measured FP64 instruction rates (the FP64 sweeps' ALU roofline)
    fp64_rate = measure_fp64_peak(aar, stream, local)

    # ---- plain FP64 form
    plain = None
    if args.plain_steps > 0:
        x_mixed = x.clone()  # the mixed form's solution, for its error against the FP64 form
        fp64 = aar.Solver.stencil(desc, aar.FP64, stream=stream)
        with torch.cuda.stream(stream):
            r0 = fp64.solve(b, x, prm=prm)
            torch.cuda.synchronize()
            q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            for _ in range(args.plain_steps):
                r0 = fp64.solve(b, x, prm=prm)
            q1.record(stream)
            torch.cuda.synchronize()
        plain_ms = q0.elapsed_time(q1) / args.plain_steps
        sweep64 = fp64.profile_kernel(aar.K_SWEEP, 5)
        # FP64 instructions per point of the radius-r sweep: 5r sums (issued as multiply-adds with a
        # unit multiplier) and r FMAs for the stencil, the centre product, the residual (an add),
        # the scaling and the Richardson update
        n_add, n_fma = 1, 6 * RADIUS + 3
        dp_instr = n_add + n_fma
        dp_peak, pk = fp64_mix_peak(fp64_rate, n_add, n_fma)
        plain = {"solves_per_s": 1e3 / plain_ms, "ms_per_solve": plain_ms, "iterations": r0.iterations,
                 "anderson_steps": r0.anderson_steps, "status": r0.status,
                 "rel_residual": fp64.rel_residual(b, x),
                 # relative 2-norm difference between the mixed form's solution and the GPU's
                 # FP64 one (the FP64 form matches the CPU oracle to 1e-9 in the parity tests,
                 # where the mixed form's error against the oracle itself is asserted)
                 "mixed_error_vs_gpu_fp64": float(torch.linalg.vector_norm(x_mixed - x) / torch.linalg.vector_norm(x)),
                 "sweep_ms": sweep64,
                 "sweep_roofline": {"bound": "alu", "achieved": dp_instr * n / (sweep64 * 1e-3) / 1e12,
                                    "peak": dp_peak / 1e12, "unit": "TDPinstr/s", "peak_kind": pk,
                                    "frac": dp_instr * n / (sweep64 * 1e-3) / dp_peak,
                                    "hbm_gbs": 32.0 * n / (sweep64 * 1e-3) / 1e9}}
        fp64.close()

    # ---- the small 32^3 7-point FP64 workload (and one full oracle solve of it on the host)
    small = None if args.no_small else run_small_poisson(aar, torch, dev, stream,
                                                         cpu=(rank == 0 and world == 1 and not args.no_cpu_baseline))

    # ---- the 128^3 nonsymmetric CSR workload
    csr = None if args.no_csr else run_csr(aar, torch, dev, stream, fp64_rate)

    # ---- batched: 512 uneven Helmholtz systems per launch
    batched = None if args.no_batched else run_batched(aar, torch, dev, stream)

    # ---- periodic boundaries, the paper's sixth-order stencil
    periodic = None if args.no_periodic else run_periodic(aar, torch, dev, stream)

    # ---- block Jacobi (2 x 2 x 2 boxes) on the headline and periodic workloads
    block = None if args.no_block else run_block(aar, torch, dev, stream, ms_step,
                                                 periodic["mixed_ms"] if periodic else None)

    # ---- complex-valued systems: the OF-DFT Helmholtz equation (Eq. 7)
    complex_ = None if args.no_complex else run_complex(aar, torch, dev, stream,
                                                          cpu=(rank == 0 and not args.no_cpu_baseline), fp64=fp64_rate)

    # ---- complex-valued systems with block Jacobi (2 x 2 x 2 boxes)
    complex_block = None if (args.no_complex or args.no_block) else run_complex_block(aar, torch, dev, stream, complex_)

    # ---- serving: continuous batching of a request stream
    serve = None if (args.no_serve or world > 1) else run_serving(aar, torch, stream)

    # ---- CPU oracle baseline on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        its = plain["iterations"] if plain else FP64_ITERS
        s_it = oracle_sample(P, PRM["p"])
        cpu = {"value": 1.0 / (s_it * its) if its else None, "unit": "solves/s", "cores": 1, "host": host_cores(),
               "kind": "oracle",
               "sample": f"one Anderson cycle ({PRM['p']} FP64 oracle iterations) on the full grid, "
                         f"{s_it:.2f} s/iteration, scaled by the {its} iterations this run's FP64 GPU solve took "
                         f"(the FP64 path's counts equal the oracle's in the parity tests)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": CONFIG,
            "hbm_gbs": hbm_bytes / (ms_step * 1e-3) / 1e9,
            "iterations": info.iterations, "anderson_steps": info.anderson_steps, "refinements": info.refinements,
            "rel_residual_fp64": r_true, "all_converged": ok,
            "roofline": roofline, "kernel_ms": kernel_times, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk.summary(), "plain_fp64": plain,
            "mixed_over_plain": (value / plain["solves_per_s"]) if plain else None,
            "fp64_rate": fp64_rate, "poisson_32": small, "csr_128": csr,
            "batched": batched, "periodic": periodic, "block_jacobi": block, "complex": complex_,
            "complex_block_jacobi": complex_block,
            "serve": serve,
            "p50_ms": serve["p50_ms"] if serve else None, "p99_ms": serve["p99_ms"] if serve else None,
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
