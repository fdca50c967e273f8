#!/usr/bin/env python3
"""Benchmark of the two-grid deflated Krylov solve on GB300: fine-grid solves per second
to relative residual 1e-8.

One step is one pass of the whole path over one synthetic right-hand side:
coarse GMRES-DR(m,k) (Section 2.1) on the restricted right-hand side, prolongation of
the k eigenvectors and of the coarse solution (Section 3, phase 1), A Y and its CholQR2
factorisation, then BiCGStab(ncyc)-Proj(k) (Section 4.1) on the fine grid until
||b - A x|| / ||b|| <= 1e-8 (verified in float64 by the library at exit).

Default workload (cd3d_255): -Lap u + beta . grad u on the unit cube, beta = (2, 1, 0.5),
7-point centred differences, fine grid 255^3 (16,581,375 unknowns), coarse grid 127^3,
30 eigenvectors prolonged trilinearly, b ~ N(0, 1), float64 throughout.

  python bench.py [--steps K] [--warmup W] [--workload cd3d_255|cd2d_127] [--impl tg|reference]

Prints one JSON line (rank 0).  Under torchrun with N ranks each rank solves its own
right-hand side (independent replicas: the path has no data-path exchange).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "cd3d_255": dict(kind="cd3d", N=255, beta=(2.0, 1.0, 0.5), m=60, k=30, nev=30, rtolev=1e-2, rtol_c=1e-8,
                     max_cycles=300, method="bicgstab", proj="minres", precision="f64", rtol=1e-8, ncyc=20,
                     restart_mvps=0, m3=20),
    # a smaller case of the same kernels for profiler captures (coarse basis 418 MB > L2)
    "cd3d_191": dict(kind="cd3d", N=191, beta=(2.0, 1.0, 0.5), m=60, k=30, nev=30, rtolev=1e-2, rtol_c=1e-8,
                     max_cycles=300, method="bicgstab", proj="minres", precision="f64", rtol=1e-8, ncyc=20,
                     restart_mvps=0, m3=20),
    # 32^4 U(1) lattice, complex128, mass tuned to lambda_min = 1e-3, coarse 16^4 Galerkin, k = 40
    "u1_32": dict(kind="u1_4d", N=32, m=80, k=40, nev=40, rtolev=1e-2, rtol_c=1e-8, max_cycles=300,
                  method="bicgstab", proj="minres", precision="f64", rtol=1e-8, ncyc=20, restart_mvps=0, m3=20),
    # the same with the moved vectors improved on the fine lattice (10 Arnoldi-E(80, 40) cycles)
    "u1_32_improved": dict(kind="u1_4d", N=32, m=80, k=40, nev=40, rtolev=1e-2, rtol_c=1e-8, max_cycles=300,
                           method="bicgstab", proj="minres", precision="f64", rtol=1e-8, ncyc=20, restart_mvps=0,
                           m3=20, improve=dict(m=80, cycles=10, nstart=10, rtolev=1e-3)),
    # 128 independent 2D problems, N_i odd ~ U{255..1023}, beta_i ~ U(0.5, 4), 8 right-hand
    # sides each sharing one 20-vector basis; float32 inner BiCGStab, float64 refinement
    # coarse phase GMRES-DR(60,20), at most 100 cycles: the whole-step optimum of a sweep over
    # (m, cycles) = (40, 300), (60, 50), (60, 100) on these 128 instances (21.6, 56.4, 18.1 s);
    # both arms use it
    "batch128": dict(kind="batch", count=128, m=60, k=20, nev=20, rtolev=1e-2, rtol_c=1e-8, max_cycles=100,
                     method="bicgstab", proj="minres", precision="f32_ir", rtol=1e-8, ncyc=20, restart_mvps=0,
                     threads=32),
    # a 16-instance cut of the batched workload (same size range) for profiler captures
    "batch16": dict(kind="batch", count=16, m=60, k=20, nev=20, rtolev=1e-2, rtol_c=1e-8, max_cycles=100,
                    method="bicgstab", proj="minres", precision="f32_ir", rtol=1e-8, ncyc=20, restart_mvps=0,
                    threads=16),
    "cd2d_127": dict(kind="cd2d", N=127, beta=(1.0,), m=30, k=15, nev=15, rtolev=1e-4, rtol_c=1e-8,
                     max_cycles=300, method="bicgstab", proj="minres", precision="f64", rtol=1e-8, ncyc=0,
                     restart_mvps=60, m3=20),
}
# The paper's own experiments (loose comparison of matrix-vector product counts; not timed
# headline workloads): Example 1 / 2 (Tables 3.1, 4.1) and Example 4 (Helmholtz).  The coarse
# grid is reached by chaining the library's factor-2 levels (bilinear prolongations compose to
# the bilinear interpolation from the coarsest grid, since the grids nest).
PAPER_RUNS = {
    "ex1_511": dict(kind="exp2d", beta=(40.0, 40.0, 5.0), mass=None, N=511, coarse_N=63, m=150, k=100, nev=80,
                    rtolev=1e-8, rtol_c=1e-10, max_cycles=400, rtol=1e-10, rhs="example1", proj="galerkin",
                    bicg_ncyc=[5, 10, 15, 20, 30, 50, 100, 150, 200], gmres_m3=[50, 100, 200], idr_ncyc=[20],
                    coarse_sweep=[127, 31, 15],
                    paper={"coarse_cycles_eig": 107, "coarse_mvps_eig": 5450, "coarse_cycles_linear": 19,
                           "table_4_1_mvps": {"5": 9638, "10": 7606, "15": 6390, "20": 5421, "30": 5357, "50": 5278,
                                              "100": 5262, "150": 5591, "200": 5541},
                           "table_4_1_cycles_used": {"100": 99, "150": 140, "200": 168},
                           "table_3_1_fine_cycles_gmres100": {"255": 85, "127": 86, "63": 94, "31": 106, "15": 120,
                                                              "7": 177, "none": 1255},
                           "table_3_1_coarse_cycles": {"255": 1023, "127": 270, "63": 107, "31": 43, "15": 12}}),
    "helm_511": dict(kind="cd2d", beta=(0.0,), mass=-1e4, N=511, coarse_N=127, m=200, k=150, nev=120, rtolev=1e-8,
                     rtol_c=1e-10, max_cycles=400, rtol=1e-10, rhs="random", proj="galerkin", interp="cubic",
                     bicg_ncyc=[20], gmres_m3=[100], idr_ncyc=[20], coarse_sweep=[],
                     paper={"coarse_cycles_eig": 285, "note": "GMRES(100)-Proj(150) and IDR(20)-Proj(150) converge; "
                                                              "IDR(20)-Proj(150) is the fastest; plain IDR does not "
                                                              "converge (Figure 5.1, counts not printed)"}),
}
# the same experiments with the other interpolation (the paper generally uses splines; the
# cubic interpolation stands in for them, bilinear is the default of the library)
PAPER_RUNS["helm_511_linear"] = dict(PAPER_RUNS["helm_511"], interp="linear")
PAPER_RUNS["ex1_511_cubic"] = dict(PAPER_RUNS["ex1_511"], interp="cubic", coarse_sweep=[])
L2_BYTES = 129 * 1024 * 1024
FP64_PEAK_TFLOPS = 152 * 4 * 2070e6 / 1e12     # 152 SMs x 2 FP64 FMA/clk x 2 flops per FMA x 2070 MHz
NOMINAL_HBM_GBS = 8000.0                         # the ~8 TB/s nominal HBM3e figure the 70% target refers to
# DRAM bytes (read + write) per launch over algorithmic bytes per launch, per kernel class,
# from an ncu capture of a smaller case of the same kernel (profiles/gemv_t_pipe_cd3d191.md:
# k_gemv_t_pipe<double>, (150.95 + 3.6) MB over 150.9 MB);
# the traffic of a full-size launch is this ratio times its algorithmic bytes (the traffic
# grows in proportion to rows x columns).  Remove an entry when its kernel changes.
NCU_TRAFFIC_RATIO = {"gemv_t": 1.024}


def dgemm_tflops(dev, n=4096, reps=5):
    """cuBLAS float64 GEMM rate on this GPU (torch.matmul), measured with CUDA events: the
    attainable float64 rate beside the derived FP64 peak (context for the ALU-bound kernels)."""
    import torch
    try:
        a = torch.randn(n, n, dtype=torch.float64, device=dev)
        b = torch.randn(n, n, dtype=torch.float64, device=dev)
        for _ in range(2):
            torch.matmul(a, b)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        del a, b
        return round(reps * 2.0 * n ** 3 / t / 1e12, 4)
    except Exception:
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, device_id: str):
        self.device_id = device_id
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", "-i", self.device_id, "--query-gpu=" + ",".join(self.FIELDS),
               "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.samples.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                mhz.append(float(s[0]))
                mx = float(s[1])
            except ValueError:
                continue
            for name, v in zip(names, s[3:]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz)}


# ----------------------------------------------------------------------------- lattice input
def lattice_operator(tg, L, seed=0, lam_min=1e-3, iters=200):
    """The lattice workload's operator: links from the seeded generator and the mass that
    puts the smallest eigenvalue at lam_min.  lambda_max of the hopping term D comes from
    plain Lanczos whose products are the library's own operator (mass -8 gives -D);
    input preparation, outside any timed region."""
    import numpy as np
    import torch

    import tg_inputs as gi
    links = torch.from_numpy(gi.u1_links(L, seed)).cuda()
    op0 = tg.Operator("u1_4d", L, links=links, mass=-8.0)
    g = torch.Generator(device="cpu").manual_seed(seed)
    V = L ** 4
    q = torch.complex(torch.randn(V, generator=g, dtype=torch.float64),
                      torch.randn(V, generator=g, dtype=torch.float64)).cuda()
    q /= torch.linalg.vector_norm(q)
    qprev = torch.zeros_like(q)
    alpha, betas, b = [], [], 0.0
    for _ in range(iters):
        w = -op0.apply(q)
        a = torch.vdot(q, w).real.item()
        w = w - a * q - b * qprev
        alpha.append(a)
        b = torch.linalg.vector_norm(w).item()
        betas.append(b)
        qprev, q = q, w / b
    T = np.diag(alpha) + np.diag(betas[:-1], 1) + np.diag(betas[:-1], -1)
    mass = float(np.linalg.eigvalsh(T)[-1] - 8.0 + lam_min)
    return tg.Operator("u1_4d", L, links=links, mass=mass), mass


# ----------------------------------------------------------------------------- GPU arm
# ----------------------------------------------------------------------------- ranks
def rank_barrier(world, dev):
    """All ranks meet, then the device is idle (the timed region's bracket)."""
    import torch
    if world > 1:
        torch.distributed.barrier()
    if dev.type == "cuda":
        torch.cuda.synchronize(dev)


def max_over_ranks_of(v, world, dev):
    """The largest of the ranks' values (the slowest rank's time)."""
    if world == 1:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_rate(units_per_rank, ms_max, world):
    """Whole-job throughput: every rank's units over the slowest rank's time (units/s)."""
    return world * units_per_rank * 1000.0 / ms_max


def run_tg(args, wl, rank, world):
    import numpy as np
    import torch

    import tg_inputs as gi
    from paper_2005_03070_gb300 import build as tgbuild
    tgbuild.build()
    from paper_2005_03070_gb300 import tg

    dev = torch.device("cuda", torch.cuda.current_device())
    if wl["kind"] == "u1_4d":
        op, mass = lattice_operator(tg, wl["N"], seed=rank)
        wl = dict(wl, mass=mass)
        b_host = torch.from_numpy(gi.rhs(op.n, seed=rank).astype(np.complex128)).pin_memory()
    else:
        op = tg.Operator(wl["kind"], wl["N"], wl["beta"])
        b_host = torch.from_numpy(gi.rhs(op.n, seed=rank)).pin_memory()
    n = op.n
    b = b_host.to(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev) if n * 8 < L2_BYTES else None

    def step(bvec, precision, mid=None):
        xc, defl, cst, _ = op.coarse_gmresdr(bvec, wl["m"], wl["k"], nev=wl["nev"], rtolev=wl["rtolev"],
                                            rtol=wl["rtol_c"], max_cycles=wl["max_cycles"], proj=wl["proj"],
                                            precision=precision)
        x = op.prolong(xc)
        if wl.get("improve"):
            # the paper's optional phase 2: Arnoldi-E cycles on the moved vectors (fine grid)
            im = wl["improve"]
            defl.improve(m=im["m"], cycles=im["cycles"], nstart=im["nstart"], nev=wl["nev"], rtolev=im["rtolev"])
        if mid is not None:
            mid.record(torch.cuda.current_stream())     # end of the setup (coarse phase, A Y, factor[, improve])
        status, st = op.solve(bvec, x, defl, method=wl["method"], precision=precision, rtol=wl["rtol"],
                              ncyc=wl["ncyc"], restart_mvps=wl["restart_mvps"], m3=wl["m3"])
        return x, status, st[0], cst

    def timed_steps(K, precision, host_io=False, profile=False):
        """K steps timed with CUDA events on the current stream (each step bracketed, the
        L2 flushed between steps when the inputs fit in L2)."""
        stream = torch.cuda.current_stream()
        total_ms = 0.0
        setup_ms = 0.0
        infos = []
        x_host = torch.empty(n, dtype=op.dtype).pin_memory() if host_io else None
        if profile:
            tg.tg_profile_enable(True)
        l0 = tg.tg_launch_count()
        for _ in range(K):
            if flush is not None:
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            em = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if host_io:
                bd = b_host.to(dev, non_blocking=True)
                x, status, st, cst = step(bd, precision, em)
                x_host.copy_(x, non_blocking=True)
            else:
                x, status, st, cst = step(b, precision, em)
            e1.record(stream)
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1)
            setup_ms += e0.elapsed_time(em)
            infos.append((status, st, cst))
        launches = tg.tg_launch_count() - l0
        prof = None
        if profile:
            prof = tg.tg_profile_read()
            tg.tg_profile_enable(False)
        split[precision] = (setup_ms / K, (total_ms - setup_ms) / K)
        return total_ms / K, infos, launches, prof

    split = {}      # precision -> (setup ms, fine-solve ms) per step of the last timed run

    def barrier():
        rank_barrier(world, dev)

    def max_over_ranks(v):
        return max_over_ranks_of(v, world, dev)

    # warm-up (also allocates every workspace)
    for _ in range(args.warmup):
        step(b, wl["precision"])
    torch.cuda.synchronize()

    dev_id = str(getattr(torch.cuda.get_device_properties(dev), "uuid", "") or "")
    dev_id = ("GPU-" + dev_id) if dev_id and not dev_id.startswith("GPU-") else (dev_id or str(dev.index))
    clocks = ClockSampler(dev_id)
    clocks.start()
    barrier()
    # the headline: the product path as a user runs it (no per-launch instrumentation, the
    # coarse cycles replayed as CUDA graphs)
    ms, infos, launches, _ = timed_steps(args.steps, wl["precision"])
    barrier()
    clocks.stop()
    ms = max_over_ranks(ms)
    setup_ms, fine_ms = (max_over_ranks(v) for v in split[wl["precision"]])
    ok = all(s == tg.TG_OK and st["relres"] <= wl["rtol"] for s, st, _ in infos)
    k_side = max(1, min(args.steps, args.side_steps))

    # end to end through the public API with host buffers (H2D of b, D2H of x per step)
    barrier()
    ms_e2e, infos_e2e, _, _ = timed_steps(k_side, wl["precision"], host_io=True)
    barrier()
    ms_e2e = max_over_ranks(ms_e2e)

    # the float32 + float64 refinement form of the same workload
    ms_ir = None
    ir_ok = None
    if wl["kind"] != "u1_4d" and not args.no_ir:
        for _ in range(1):
            step(b, "f32_ir")
        barrier()
        ms_ir, infos_ir, _, _ = timed_steps(k_side, "f32_ir")
        barrier()
        ms_ir = max_over_ranks(ms_ir)
        setup_ir, fine_ir = (max_over_ranks(v) for v in split["f32_ir"])
        ir_ok = all(s == tg.TG_OK and st["relres"] <= wl["rtol"] for s, st, _ in infos_ir)

    # GMRES(m3)-Proj on the same workload (the 3D configuration compares it with BiCGStab-Proj)
    gmres = None
    if wl["kind"] == "cd3d" and not args.no_gmres:
        wg = dict(wl, method="gmres")
        wl_saved = dict(wl)
        wl.update(wg)
        step(b, wl["precision"])
        barrier()
        ms_g, infos_g, _, _ = timed_steps(min(k_side, 2), wl["precision"])
        barrier()
        ms_g = max_over_ranks(ms_g)
        setup_g, fine_g = (max_over_ranks(v) for v in split[wl["precision"]])
        wl.clear()
        wl.update(wl_saved)
        sg = infos_g[-1][1]
        gmres = {"method": f"GMRES({wl['m3']})-Proj({wl['k']})", "value": round(world * 1000.0 / ms_g, 5),
                 "unit": "solves/s", "ms_per_step": round(ms_g, 3),
                 "converged": all(s_ == tg.TG_OK and st_["relres"] <= wl["rtol"] for s_, st_, _ in infos_g),
                 "fine_solve_ms": round(fine_g, 3), "fine_mvps": sg["mvps"], "fine_cycles": sg["cycles"],
                 "fine_solve_only": round(world * 1000.0 / fine_g, 5),
                 "bicgstab_fine_solve_ms": round(fine_ms, 3)}

    # per-kernel-class profile: one more step with a CUDA event pair around every launch
    # (eager launches, no graph replay), outside the timed regions above
    _, _, _, prof = timed_steps(1, wl["precision"], profile=True)
    prof_ir = None
    if ms_ir is not None:
        _, _, _, prof_ir = timed_steps(1, "f32_ir", profile=True)
        prof_ir.pop("gmresdr_restart_phase_cycles", None)

    status, st, cst = infos[-1]
    phases = prof.pop("gmresdr_restart_phase_cycles", None)
    peaks, peak_src = measured_peaks()
    # roofline of the dominant kernel class (largest share of device time in the timed region)
    dom_name, dom = max(((k, v) for k, v in prof.items() if k != "bicg_noop"), key=lambda kv: kv[1]["ms"])
    dev_ms_total = sum(v["ms"] for v in prof.values())
    per_launch_ms = dom["ms"] / dom["launches"]
    gbs = dom["bytes"] / (dom["ms"] * 1e-3) / 1e9
    tflops = dom["flops"] / (dom["ms"] * 1e-3) / 1e12
    ratio = NCU_TRAFFIC_RATIO.get(dom_name)
    traffic = None if ratio is None else ratio * dom["bytes"] / dom["launches"]
    dgemm = dgemm_tflops(dev)
    roofline = {"kernel": dom_name, "bound": "alu", "achieved": round(tflops, 4),
                "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s", "frac": round(tflops / FP64_PEAK_TFLOPS, 4),
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops per FMA x 2070 MHz",
                "fp64_dgemm_tflops_measured": dgemm,
                "frac_of_dgemm": round(tflops / dgemm, 4) if dgemm else None,
                "traffic": traffic, "algorithmic_bytes_per_launch": dom["bytes"] / dom["launches"],
                "algorithmic_flops_per_launch": dom["flops"] / dom["launches"],
                "ms_per_launch": round(per_launch_ms, 5), "hbm_gbs": round(gbs, 1),
                "hbm_frac": round(gbs / peaks["hbm_gbs"], 4), "hbm_peak_gbs": peaks["hbm_gbs"],
                "hbm_peak_source": peak_src, "share_of_device_time": round(dom["ms"] / dev_ms_total, 4)}
    kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                   "share": round(v["ms"] / dev_ms_total, 4),
                   "gbs": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1) if v["ms"] > 0 else 0.0,
                   "tflops": round(v["flops"] / (v["ms"] * 1e-3) / 1e12, 4) if v["ms"] > 0 else 0.0}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:10]}
    target_classes = class_rooflines(prof, prof_ir, peaks["hbm_gbs"])
    value = weak_scaling_rate(1, ms, world)
    line = {
        "metric": "fine-grid solves/sec to rel. residual 1e-8 (FP64 vs batched FP32+IR) and HBM GB/s",
        "value": round(value, 5), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128" if wl["kind"] == "u1_4d" else "f64",
        "data": "synthetic (seeded N(0,1) right-hand side)",
        "config": {"workload": args.workload, **{k: (list(v) if isinstance(v, tuple) else v) for k, v in wl.items()},
                   "n": n, "n_coarse": op.nc,
                   "l2": "inputs larger than L2" if flush is None else "L2 flushed between steps",
                   "parallelism": f"replicas x{world}"},
        "solves_converged": ok,
        "step_breakdown": {"coarse_cycles": cst["cycles"], "coarse_mvps": cst["coarse_mvps"],
                           "eig_converged": cst["eig_converged"], "fine_mvps": st["mvps"],
                           "fine_cycles": st["cycles"], "relres": st["relres"]},
        # the step split at the end of the set-up (coarse GMRES-DR, prolongation, A Y and its
        # factorisation) and the fine solve from the prolonged x_0; the set-up is shared by every
        # right-hand side that uses the same operator, so the fine-solve rate is reported too
        "step_phases_ms": {"setup": round(setup_ms, 3), "fine_solve": round(fine_ms, 3)},
        "fine_solve_only": {"value": round(world * 1000.0 / fine_ms, 5), "unit": "solves/s",
                            "note": "set-up excluded (amortised over right-hand sides)"},
        "e2e": {"value": round(world * 1000.0 / ms_e2e, 5), "unit": "solves/s",
                "h2d_bytes_per_step": n * b_host.element_size(), "d2h_bytes_per_step": n * b_host.element_size()},
        "gmres_proj": gmres,
        "fp32_ir": None if ms_ir is None else {"value": round(world * 1000.0 / ms_ir, 5), "unit": "solves/s",
                                               "ms_per_step": round(ms_ir, 3), "converged": ir_ok,
                                               "speedup_vs_f64": round(ms / ms_ir, 3),
                                               "step_phases_ms": {"setup": round(setup_ir, 3),
                                                                  "fine_solve": round(fine_ir, 3)},
                                               "fine_solve_only": round(world * 1000.0 / fine_ir, 5),
                                               "fine_solve_speedup_vs_f64": round(fine_ms / fine_ir, 3)},
        "gpu_launches": int(launches),
        "roofline": roofline,
        # the three kernel classes the 70%-of-HBM target names (stencil, BiCGStab update,
        # projection), in both precisions; float64 ones are FP64-ALU bound on this GPU
        "roofline_target_classes": target_classes,
        "kernels": kernels,
        "profile_note": "kernels / roofline from one extra step per precision with CUDA events around every "
                        "launch (eager launches), outside the timed regions",
        "gmresdr_restart_phase_us": None if not phases else
            [round(p / max(1, cst["cycles"]) / 2070.0, 1) for p in phases],
        "clocks": clocks.summary(),
    }
    return line, {"coarse_cycles": cst["cycles"], "fine_mvps": st["mvps"], "fine_cycles": st["cycles"],
                  "coarse_steps": cst["coarse_mvps"]}


def class_rooflines(prof64, prof32, hbm_peak):
    """Achieved HBM rate of the stencil, BiCGStab-update and projection kernel classes
    (algorithmic bytes / CUDA-event time), against the measured copy peak and against the
    nominal 8 TB/s, and the FP64 rate against the FP64 ALU peak."""
    groups = {"stencil": ("bicg_v", "bicg_t"), "bicgstab_update": ("bicg_x", "bicg_s"),
              "projection": ("proj_update",)}
    out = {}
    for prec, prof in (("f64", prof64), ("f32", prof32)):
        if not prof:
            continue
        for g, names in groups.items():
            for nm in names:
                v = prof.get(nm)
                if not v or v["ms"] <= 0:
                    continue
                gbs = v["bytes"] / (v["ms"] * 1e-3) / 1e9
                e = {"launches": v["launches"], "us_per_launch": round(1e3 * v["ms"] / v["launches"], 2),
                     "gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 4),
                     "hbm_frac_nominal": round(gbs / NOMINAL_HBM_GBS, 4)}
                if prec == "f64":
                    tf = v["flops"] / (v["ms"] * 1e-3) / 1e12
                    e["fp64_tflops"] = round(tf, 4)
                    e["fp64_frac"] = round(tf / FP64_PEAK_TFLOPS, 4)
                out[f"{g}.{nm}.{prec}"] = e
    return out


# ----------------------------------------------------------------------------- oracle arm
def _timeit(f, min_time=0.5, max_reps=20):
    """Seconds per call of f after one untimed call, averaged over >= min_time."""
    f()
    reps, t0 = 0, time.perf_counter()
    while True:
        f()
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_time or reps >= max_reps:
            return el / reps


class CpuPieces:
    """The oracle (numpy FP64, as it stands) on bounded pieces of the workload, and the
    scaling of the pieces' times to one full solve with the given step counts."""

    def __init__(self, wl, counts):
        import numpy as np

        import tg_inputs as gi
        from oracle import transfer as otr
        from oracle.operators import CD2D, CD3D, Operator, coarse_operator
        kind = {"cd2d": CD2D, "cd3d": CD3D}[wl["kind"]]
        self.wl, self.counts = wl, counts
        self.op = Operator(kind, wl["N"], wl["beta"])
        self.opc = coarse_operator(self.op)
        self.n, self.k = self.op.n, wl["k"]
        self.b = gi.rhs(self.n, 0)
        self.bc = otr.restrict(self.b, wl["N"], 2 if wl["kind"] == "cd2d" else 3)
        self.np = np
        # projection: for large n it is timed at two smaller widths k1 < k2 and extrapolated
        # with t(k) = a k + c k^2 (products linear in k, the QR quadratic)
        if self.n * self.k <= 50_000_000:
            self.widths = (self.k,)
        else:
            self.widths = (max(2, self.k // 5), max(4, (2 * self.k) // 5))
        self.names = ["fine_iter", "fine_mvp"] + [f"projection_{w}" for w in self.widths] + \
                     ["coarse_cycles_1", "coarse_cycles_2"]
        self.times = {nm: [] for nm in self.names}

    def run(self, name):
        """Time one piece once (seconds), record it."""
        import tg_inputs as gi
        from oracle import gmresdr as ogd
        from oracle import krylov
        np, wl, n = self.np, self.wl, self.n
        t0 = time.perf_counter()
        if name == "fine_iter":          # one BiCGStab iteration: 2 products and its updates
            krylov.bicgstab_cycle(self.op.apply, np.zeros(n), self.b, 0.0, max_mvps=2)
        elif name == "fine_mvp":
            self.op.apply(self.b)
        elif name.startswith("projection_"):
            kw = int(name.split("_")[1])
            d = krylov.Deflation(gi.random_dense((n, kw), 1), gi.random_dense((n, kw), 2), wl["proj"])
            t0 = time.perf_counter()
            krylov.project(d, np.zeros(n), self.b.copy())
        else:                            # whole oracle GMRES-DR runs of one and of two cycles
            cyc = int(name[-1])
            ogd.gmresdr(self.opc.apply, self.bc, wl["m"], wl["k"], nev=wl["nev"], rtolev=wl["rtolev"],
                        rtol=wl["rtol_c"], max_cycles=cyc)
        dt = time.perf_counter() - t0
        self.times[name].append(dt)
        return dt

    def estimate(self):
        """Seconds per full solve from the median time of each piece."""
        med = {k: statistics.median(v) for k, v in self.times.items() if v}
        k, c = self.k, self.counts
        if len(self.widths) == 1:
            t_proj = med[f"projection_{k}"]
        else:
            k1, k2 = self.widths
            t1, t2 = med[f"projection_{k1}"], med[f"projection_{k2}"]
            cq = (t2 / k2 - t1 / k1) / (k2 - k1)
            a_ = t1 / k1 - cq * k1
            t_proj = max(a_ * k + cq * k * k, t2 * k / k2)
        t_c1 = med["coarse_cycles_1"]
        t_cycle = max(med["coarse_cycles_2"] - t_c1, 0.0)
        est = (t_c1 + (c["coarse_cycles"] - 1) * t_cycle + k * med["fine_mvp"]
               + c["fine_mvps"] / 2 * med["fine_iter"] + c["fine_cycles"] * (t_proj + med["fine_mvp"]))
        return est, {"fine_iter": med["fine_iter"], "fine_mvp": med["fine_mvp"], "projection": t_proj,
                     "coarse_cycle1": t_c1, "coarse_cycle": t_cycle}

    def info(self, est, pieces, samples, wall):
        try:
            from threadpoolctl import threadpool_info
            blas = max([p.get("num_threads", 1) for p in threadpool_info()] + [1])
        except Exception:
            blas = os.cpu_count() or 1
        w = self.widths
        proj_note = (f"one {w[0]}-vector MinRes projection" if len(w) == 1 else
                     f"MinRes projections with {w[0]} and {w[1]} vectors (extrapolated to {self.k} as a k + c k^2)")
        c = self.counts
        return {"kind": "oracle", "cores": blas,
                "cores_note": f"stencil and vector steps run on 1 core; BLAS/LAPACK calls (projection QR, "
                              f"dense products) on {blas} threads",
                "sample": (f"oracle (numpy float64) timed on {samples} samples of bounded pieces: one fine BiCGStab "
                           f"iteration, one fine product, {proj_note}, and coarse GMRES-DR runs of one and of two "
                           f"cycles; the value is one solve extrapolated from the pieces' median times with "
                           f"{c['coarse_cycles']} coarse cycles, {self.k} A Y products, {c['fine_mvps']} fine products "
                           f"and {c['fine_cycles']} fine cycles (the oracle's own full-run counts)"),
                "samples": samples, "sample_seconds": round(wall, 2), "est_seconds_per_solve": round(est, 3),
                "pieces_s": pieces}


def cpu_sample(wl, counts):
    """Every piece once; returns (solves/s, info)."""
    t0 = time.perf_counter()
    cp = CpuPieces(wl, counts)
    for nm in cp.names:
        cp.run(nm)
    est, pieces = cp.estimate()
    return 1.0 / est, cp.info(est, pieces, len(cp.names), time.perf_counter() - t0)


def oracle_counts(workload):
    """Step counts of the oracle's own full run (written by oracle/bench_counts.py)."""
    path = os.path.join(ROOT, "oracle", "bench_counts.json")
    with open(path) as f:
        return json.load(f)[workload]


def run_batch(args, wl, rank, world, fp64_instances=0):
    """128 cd2d instances x 8 right-hand sides: the batched float32+refinement form against the per-instance
    float64 path.  fp64_instances > 0 times the float64 path on that many instances (every
    (count / fp64_instances)-th by size, all 8 right-hand sides each) instead of all of them."""
    import numpy as np
    import torch

    import tg_inputs as gi
    from paper_2005_03070_gb300 import build as tgbuild
    tgbuild.build()
    from paper_2005_03070_gb300 import tg

    dev = torch.device("cuda", torch.cuda.current_device())
    Ns, betas = gi.batch_instances(wl["count"], seed=rank)
    batch = tg.Batch(Ns, betas)
    host = np.empty(batch.total, dtype=np.float64)
    for i, N in enumerate(Ns):
        o, n = batch.offsets[i], batch.sizes[i]
        host[o:o + n * 8] = np.ascontiguousarray(gi.rhs(n, seed=1000 * rank + i, nrhs=8).T).reshape(-1)
    rhs_h = torch.from_numpy(host).pin_memory()
    rhs = rhs_h.to(dev)
    x = torch.zeros_like(rhs)
    nsolves = wl["count"] * 8

    phase = {"setup_ms": 0.0, "solve_ms": 0.0, "coarse_cycles": []}

    def batched_step(bvec, xvec):
        t0 = time.perf_counter()
        cst = batch.setup(bvec, m=wl["m"], k=wl["k"], nev=wl["nev"], rtolev=wl["rtolev"], rtol=wl["rtol_c"],
                          max_cycles=wl["max_cycles"], proj=wl["proj"], threads=wl["threads"])
        t1 = time.perf_counter()
        xvec.zero_()
        out = batch.solve(bvec, xvec, rtol=wl["rtol"], ncyc=wl["ncyc"], restart_mvps=wl["restart_mvps"],
                          threads=wl["threads"])
        t2 = time.perf_counter()
        phase["setup_ms"], phase["solve_ms"] = 1e3 * (t1 - t0), 1e3 * (t2 - t1)
        phase["coarse_cycles"] = [c["cycles"] for c in cst]
        return out

    def timed(f, K):
        ms = 0.0
        out = None
        for _ in range(K):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = f()
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        return ms / K, out

    for _ in range(args.warmup):
        batched_step(rhs, x)
    dev_id = str(getattr(torch.cuda.get_device_properties(dev), "uuid", "") or "")
    dev_id = ("GPU-" + dev_id) if dev_id and not dev_id.startswith("GPU-") else (dev_id or str(dev.index))
    clocks = ClockSampler(dev_id)
    clocks.start()
    rank_barrier(world, dev)
    l0 = tg.tg_launch_count()
    ms, (status, stats) = timed(lambda: batched_step(rhs, x), args.steps)
    launches = (tg.tg_launch_count() - l0) // max(args.steps, 1)
    rank_barrier(world, dev)
    clocks.stop()
    ms = max_over_ranks_of(ms, world, dev)
    phase_timed = dict(phase)
    phase_timed["setup_ms"] = max_over_ranks_of(phase_timed["setup_ms"], world, dev)
    phase_timed["solve_ms"] = max_over_ranks_of(phase_timed["solve_ms"], world, dev)
    ok = status == tg.TG_OK and all(s["relres"] <= wl["rtol"] for s in stats)

    def e2e_step():
        bd = rhs_h.to(dev, non_blocking=True)
        xd = torch.zeros_like(bd)
        out = batched_step(bd, xd)
        xd.cpu()
        return out
    rank_barrier(world, dev)
    ms_e2e, _ = timed(e2e_step, 1)
    rank_barrier(world, dev)
    ms_e2e = max_over_ranks_of(ms_e2e, world, dev)

    # the plain float64 path: per instance, coarse GMRES-DR then its 8 columns one by one
    sel = list(range(len(Ns)))
    if 0 < fp64_instances < len(Ns):
        by_size = sorted(sel, key=lambda i: (batch.sizes[i], i))
        stride = len(Ns) / fp64_instances
        sel = sorted(by_size[int(stride * j + stride / 2)] for j in range(fp64_instances))
    ops = [tg.Operator("cd2d", Ns[i], (betas[i],)) for i in sel]
    cols = []
    for i in sel:
        o, n = batch.offsets[i], batch.sizes[i]
        blk = rhs[o:o + n * 8].view(n, 8)
        cols.append([blk[:, q].contiguous() for q in range(8)])
    nsolves64 = 8 * len(sel)

    split64 = {"setup": 0.0, "solve": 0.0}

    def fp64_step():
        mv = 0
        good = True
        split64["setup"] = split64["solve"] = 0.0
        for i, op in enumerate(ops):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, defl, _, _ = op.coarse_gmresdr(cols[i][0], wl["m"], wl["k"], nev=wl["nev"], rtolev=wl["rtolev"],
                                              rtol=wl["rtol_c"], max_cycles=wl["max_cycles"], want_xc=False)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            for q in range(8):
                xq = torch.zeros_like(cols[i][q])
                st, s = op.solve(cols[i][q], xq, defl, rtol=wl["rtol"], ncyc=wl["ncyc"],
                                 restart_mvps=wl["restart_mvps"])
                mv += s[0]["mvps"]
                good &= st == tg.TG_OK
            torch.cuda.synchronize()
            split64["setup"] += 1e3 * (t1 - t0)
            split64["solve"] += 1e3 * (time.perf_counter() - t1)
        return good, mv
    fp64_step()       # warm-up (allocates every workspace)
    rank_barrier(world, dev)
    ms64, (ok64, mv64) = timed(fp64_step, 1)
    rank_barrier(world, dev)
    ms64 = max_over_ranks_of(ms64, world, dev)
    split64["solve"] = max_over_ranks_of(split64["solve"], world, dev)
    value = weak_scaling_rate(nsolves, ms, world)
    n_tot = int(sum(batch.sizes))
    tune = batch.tuning()
    peaks, peak_src = measured_peaks()
    iter_bytes = n_tot * 8 * 17 * 4
    iter_gbs = iter_bytes / (tune["us_per_iteration"] * 1e-6) / 1e9 if tune["us_per_iteration"] > 0 else 0.0
    line = {
        "metric": "fine-grid solves/sec to rel. residual 1e-8 (FP64 vs batched FP32+IR) and HBM GB/s",
        "value": round(value, 3), "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 2), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 inner / f64 refinement", "data": "synthetic (seeded sizes, betas, N(0,1) right-hand sides)",
        "config": {"workload": args.workload, **{k: v for k, v in wl.items() if k != "kind"},
                   "unknowns": n_tot, "right_hand_sides": nsolves, "l2": "inputs larger than L2",
                   "parallelism": f"replicas x{world}"},
        "solves_converged": ok,
        "not_converged": int(sum(1 for s in stats if s["relres"] > wl["rtol"])),
        "relres_max": max(s["relres"] for s in stats),
        "mvps_mean": round(float(np.mean([s["mvps"] for s in stats])), 1),
        "mvps_max": int(max(s["mvps"] for s in stats)),
        "step_phases_ms": {"setup": round(phase_timed["setup_ms"], 1), "solve": round(phase_timed["solve_ms"], 1),
                           "coarse_cycles_mean": round(float(np.mean(phase_timed["coarse_cycles"])), 1),
                           "coarse_cycles_max": int(max(phase_timed["coarse_cycles"]))},
        # set-up (coarse GMRES-DR, A Y, factorisations) excluded: the per-solve rate the set-up
        # is amortised against, for both forms
        "solve_only": {"value": round(world * nsolves * 1000.0 / phase_timed["solve_ms"], 3), "unit": "solves/s",
                       "fp64_per_instance": round(world * nsolves64 * 1000.0 / split64["solve"], 3),
                       "speedup_of_batched": round((nsolves / phase_timed["solve_ms"]) /
                                                   (nsolves64 / split64["solve"]), 3)},
        "e2e": {"value": round(world * nsolves * 1000.0 / ms_e2e, 3), "unit": "solves/s",
                "h2d_bytes_per_step": batch.total * 8, "d2h_bytes_per_step": batch.total * 8},
        "fp64_per_instance": {"value": round(world * nsolves64 * 1000.0 / ms64, 3), "unit": "solves/s",
                              "ms_per_step": round(ms64, 1), "converged": bool(ok64), "mvps_mean": mv64 / nsolves64,
                              "instances": len(sel), "right_hand_sides": nsolves64,
                              "sample": "all instances" if len(sel) == len(Ns) else
                                        f"{len(sel)} of {len(Ns)} instances, evenly spaced in size order",
                              "speedup_of_batched": round((world * nsolves * 1000.0 / ms) /
                                                          (world * nsolves64 * 1000.0 / ms64), 3)},
        "gpu_launches": int(launches),
        "autotuner": tune,
        # the batched BiCGStab iteration (the four phase kernels over all instances and columns):
        # algorithmic bytes 17 float32 words per point and right-hand side, over the iteration
        # time the autotuner measured with CUDA events on the batch's stream (all columns active)
        "roofline": {"kernel": "batched BiCGStab iteration (k_mrb_bi_v/s/t/x, all instances)", "bound": "hbm",
                     "achieved": round(iter_gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": round(iter_gbs / peaks["hbm_gbs"], 4),
                     "frac_nominal": round(iter_gbs / NOMINAL_HBM_GBS, 4), "peak_source": peak_src,
                     "algorithmic_bytes_per_iteration": iter_bytes, "us_per_iteration": tune["us_per_iteration"],
                     "traffic": None},
        "clocks": clocks.summary(),
    }
    return line


def run_paper(args, name, rank, world):
    """One of the paper's own experiments through the library: the coarse GMRES-DR phase, the
    move to the fine grid and the fine-grid solvers, reporting product counts beside the
    paper's (which come from MATLAB runs with spline interpolation: context, not parity)."""
    import numpy as np
    import torch

    import tg_inputs as gi
    from paper_2005_03070_gb300 import build as tgbuild
    tgbuild.build()
    from paper_2005_03070_gb300 import tg

    cfg = PAPER_RUNS[name]
    dev = torch.device("cuda", torch.cuda.current_device())
    N = cfg["N"]

    def chain(coarse_N):
        levels = [2 * coarse_N + 1]
        while levels[-1] < N:
            levels.append(2 * levels[-1] + 1)
        assert levels[-1] == N
        return levels

    ops = {}

    def op_of(Nl):
        if Nl not in ops:
            ops[Nl] = tg.Operator(cfg["kind"], Nl, cfg["beta"], mass=cfg["mass"], interp=cfg.get("interp", "linear"))
        return ops[Nl]

    if cfg["rhs"] == "example1":
        b = torch.from_numpy(gi.example1_rhs(N)).to(dev)
    else:
        b = torch.from_numpy(gi.rhs(N * N, seed=rank)).to(dev)

    def sync_time(f):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = f()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    def coarse_phase(coarse_N):
        levels = chain(coarse_N)
        bl = b
        for Nl in reversed(levels[1:]):
            bl = op_of(Nl).restrict(bl)
        top = op_of(levels[0])
        (xc, defl, cst, status), t_c = sync_time(lambda: top.coarse_gmresdr(
            bl, cfg["m"], cfg["k"], nev=cfg["nev"], rtolev=cfg["rtolev"], rtol=cfg["rtol_c"],
            max_cycles=cfg["max_cycles"], proj=cfg["proj"]))
        Y = defl.copy(0).reshape(-1)
        x0 = top.prolong(xc)
        kk = defl.kk
        for Nl in levels[1:]:
            Y = op_of(Nl).prolong(Y)
            x0 = op_of(Nl).prolong(x0)
        fine = op_of(N)
        # float32 copies too: the float32 + refinement IDR below uses them
        dfl, t_f = sync_time(lambda: fine.defl_from_basis(Y, kk, proj=cfg["proj"], precision="f32_ir"))
        return x0, dfl, {"coarse_N": coarse_N, "cycles": cst["cycles"], "coarse_mvps": cst["coarse_mvps"],
                         "eig_converged": cst["eig_converged"], "kk": kk, "coarse_seconds": round(t_c, 3),
                         "AY_and_factor_seconds": round(t_f, 3)}

    fine = op_of(N)
    x0, dfl, coarse = coarse_phase(cfg["coarse_N"])
    out = {"experiment": name, "coarse": coarse, "bicgstab_proj": {}, "gmres_proj": {}, "idr_proj": {}}

    def record(key, tag, fn):
        x = x0.clone()
        (status, st), t = sync_time(lambda: fn(x))
        out[key][str(tag)] = {"status": int(status), "mvps": int(st[0]["mvps"]), "cycles": int(st[0]["cycles"]),
                              "relres": st[0]["relres"], "seconds": round(t, 3)}

    for ncyc in cfg["bicg_ncyc"]:
        record("bicgstab_proj", ncyc, lambda x: fine.solve(b, x, dfl, rtol=cfg["rtol"], ncyc=ncyc, restart_mvps=0,
                                                           max_mvps=200000))
    for m3 in cfg["gmres_m3"]:
        record("gmres_proj", m3, lambda x: fine.solve(b, x, dfl, method="gmres", rtol=cfg["rtol"], m3=m3,
                                                      max_mvps=200000))
    P = torch.from_numpy(gi.random_dense((4, fine.n), 60)).to(dev)
    for ncyc in cfg["idr_ncyc"]:
        record("idr_proj", ncyc, lambda x: fine.solve_idr(b, x, P, dfl, rtol=cfg["rtol"], ncyc=ncyc,
                                                          max_mvps=200000))
    out["idr_proj_f32_ir"] = {}
    for ncyc in cfg["idr_ncyc"]:
        record("idr_proj_f32_ir", ncyc, lambda x: fine.solve_idr(b, x, P, dfl, rtol=cfg["rtol"], ncyc=ncyc,
                                                                 max_mvps=200000, precision="f32_ir"))
    # without deflation: restarted BiCGStab with one cycle (non-restarted) from x0 = 0
    xz = torch.zeros_like(b)
    (status, st), t = sync_time(lambda: fine.solve(b, xz, None, rtol=cfg["rtol"], ncyc=1, restart_mvps=0,
                                                   max_mvps=200000))
    out["bicgstab_no_deflation"] = {"status": int(status), "mvps": int(st[0]["mvps"]), "seconds": round(t, 3)}
    # Table 3.1: the coarse grid size, with GMRES(100)-Proj(k) on the fine grid
    sweep = {}
    for cN in cfg["coarse_sweep"]:
        xs, ds, cs = coarse_phase(cN)
        (status, st), t = sync_time(lambda: fine.solve(b, xs, ds, method="gmres", rtol=cfg["rtol"], m3=100,
                                                       max_mvps=400000))
        sweep[str(cN)] = {**cs, "fine_cycles": int(st[0]["cycles"]), "fine_mvps": int(st[0]["mvps"]),
                          "status": int(status), "fine_seconds": round(t, 3)}
    if sweep:
        sweep[str(cfg["coarse_N"])] = {**coarse, "fine_cycles": out["gmres_proj"].get("100", {}).get("cycles"),
                                       "fine_mvps": out["gmres_proj"].get("100", {}).get("mvps")}
        out["coarse_size_sweep_gmres100"] = sweep
    out["paper"] = cfg["paper"]
    out["config"] = {k: (list(v) if isinstance(v, tuple) else v) for k, v in cfg.items() if k != "paper"}
    return out


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--workload", default="cd3d_255", choices=sorted(WORKLOADS) + sorted(PAPER_RUNS))
    p.add_argument("--impl", default="tg", choices=["tg", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-ir", action="store_true")
    p.add_argument("--side-steps", type=int, default=5,
                   help="timed steps of the e2e and float32 side measurements (at most --steps)")
    p.add_argument("--no-batch", action="store_true", help="skip the batched-form key of the default run")
    p.add_argument("--no-gmres", action="store_true", help="skip the GMRES(m3)-Proj key of the 3D workload")
    args = p.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.workload in PAPER_RUNS:
        out = run_paper(args, args.workload, rank, world)
        if rank == 0:
            print(json.dumps(out))
        return
    wl = WORKLOADS[args.workload]

    if args.impl == "reference":
        if rank != 0:
            return
        counts = oracle_counts(args.workload)
        cp = CpuPieces(wl, counts)
        # warm-up: every piece once (the estimate needs each at least once; these samples count)
        for nm in cp.names:
            cp.run(nm)
        # K timed samples, one bounded piece each, in rotation
        t0 = time.perf_counter()
        walls = []
        for i in range(args.steps):
            walls.append(cp.run(cp.names[i % len(cp.names)]))
        wall = time.perf_counter() - t0
        est, pieces = cp.estimate()
        value = 1.0 / est
        info = cp.info(est, pieces, args.steps, wall)
        line = {"impl": "reference",
                "metric": "fine-grid solves/sec to rel. residual 1e-8 (FP64 vs batched FP32+IR) and HBM GB/s",
                "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(1000.0 * wall / max(args.steps, 1), 3),
                "step_note": "a step is one timed sample of one bounded piece of the solve; value is the full solve "
                             "extrapolated from the pieces (est_seconds_per_solve), not 1000 / ms_per_step",
                "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded N(0,1) right-hand side)",
                "config": {"workload": args.workload, **{k: (list(v) if isinstance(v, tuple) else v)
                                                        for k, v in wl.items()}},
                "cpu_baseline": {**info, "value": value, "unit": "solves/s"},
                "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "sample_wall_s": round(wall, 2)}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    if wl["kind"] == "batch":
        line = run_batch(args, wl, rank, world)
        if rank == 0:
            print(json.dumps(line))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    line, counts = run_tg(args, wl, rank, world)
    if args.workload == "cd3d_255" and not args.no_batch:
        # the batched half of the metric: 128 instances x 8 right-hand sides, batched float32 +
        # refinement against the plain per-instance float64 path (one warm-up, one timed step)
        import gc
        gc.collect()
        torch.cuda.empty_cache()
        bl = run_batch(argparse.Namespace(steps=1, warmup=1, workload="batch128"), WORKLOADS["batch128"],
                       rank, world, fp64_instances=16)
        line["batch128"] = {k: bl[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup", "solves_converged",
                                               "not_converged", "relres_max", "mvps_mean", "step_phases_ms",
                                               "solve_only", "e2e", "fp64_per_instance", "gpu_launches", "autotuner",
                                               "roofline", "clocks")}
        line["batch128"]["config"] = bl["config"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline and wl["kind"] in ("cd2d", "cd3d"):
        v, info = cpu_sample(wl, counts)
        line["cpu_baseline"] = {**info, "value": v, "unit": "solves/s"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
