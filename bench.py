#!/usr/bin/env python
"""Throughput of the compact third-order GKS hot path on GB300, in Mcell-steps/s.

Workload: the 2D Euler smooth wave of Section 4.1's analogue on the periodic square
[0, 2]^2 at 512 x 512 cells (rho = 1 + 0.2 sin(pi (x + y) + phi), U = V = 1, p = 1,
gamma = 1.4, CFL 0.5, seeded phi), the largest grid of its convergence sweep.  One
step = compact reconstruction + face evolution on every x- and y-face + conservative
update with the ghost fill + CFL dt reduction, all in the library's CUDA kernels.

The headline form is FP32-bulk (everything in FP32, the cell averages kept as
double-float hi + lo pairs updated with compensated arithmetic); the plain FP64 form
and the L1 density difference between the two are reported in the same line.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on the
solver's stream, with a 256 MiB write between steps to flush L2 (the state is smaller
than L2).  Under torchrun each rank advances its own grid (replicas; no collective on
the data path) and the max over ranks is used.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mcell-steps/s on one GB300, FP32/batched form vs plain FP64, at stated L1 error"
UNIT = "Mcell-steps/s"
N_GRID = 512
CFL = 0.5
SEED = 2
L2_FLUSH_BYTES = 256 << 20
FP32_LANES_PER_SM = 128   # FP32 FMA lanes per Blackwell SM
SM_COUNT = 152
ISSUE_PER_SM_CLK = 4      # warp instructions issued per SM per clock (four schedulers)
SM_MAX_MHZ = 2070.0


def workload_config(n=N_GRID):
    return {"workload": f"2D Euler smooth wave {n}x{n}, periodic [0,2]^2, gamma 1.4, CFL {CFL}, seed {SEED}",
            "grid": [n, n], "cells": n * n, "cfl": CFL, "tau_eps": 0.0,
            "l2": "flushed between timed steps (256 MiB write); state < L2"}


def dist_env():
    from paper_1412_4489_gb300 import parallel
    return parallel.rank_env()


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9 and f[1].replace(".", "").isdigit():
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "samples": len(rows),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def profile_figure(precision_name, key):
    """A per-face figure of the x-face kernel (`key: value` line) from the committed ncu
    summary, or None when it is missing or the kernel sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"step_kernels_{precision_name}_smooth_wave_2048.md")
    if not os.path.exists(path):
        return None, None
    h = source_hash()
    value, ok = None, False
    for line in open(path):
        if line.startswith("source_sha1:"):
            ok = line.split(":", 1)[1].strip() == h
        if line.startswith(key + ":"):
            value = float(line.split(":", 1)[1])
    return (value if ok else None), path


def flux_traffic(precision_name):
    """DRAM bytes per face of the x-face kernel (ncu), or None (see profile_figure)."""
    return profile_figure(precision_name, "traffic_bytes_per_face")


def source_hash():
    m = hashlib.sha1()
    for p in ("paper_1412_4489_gb300/csrc/gks_device.cuh", "paper_1412_4489_gb300/csrc/gks_grid.cuh",
              "paper_1412_4489_gb300/csrc/gks.cu"):
        m.update(open(os.path.join(ROOT, p), "rb").read())
    return m.hexdigest()


def face_inputs(p):
    """A representative x-face of the workload's initial state (face-frame inputs for the op count)."""
    import numpy as np
    g = p.gamma
    dx = p.Lx / p.nx
    phi = p.meta["phi"]
    x0, y0 = dx * 10, dx * 10.5

    def rho(x, y):
        return 1 + 0.2 * math.sin(math.pi * (x + y) + phi)

    def cons(r):
        return np.array([r, r, r, 1 / (g - 1) + r])

    h = 1e-4
    S = np.zeros((6, 4))
    S[0] = cons(rho(x0, y0))
    dr = (rho(x0 + h, y0) - rho(x0 - h, y0)) / (2 * h)
    ddr = (rho(x0 + h, y0) - 2 * rho(x0, y0) + rho(x0 - h, y0)) / h ** 2
    # rho U = rho V = rho and rho E = 1/(g-1) + rho share the derivatives of rho
    S[1] = S[2] = dr
    S[3] = S[4] = S[5] = ddr
    avg = np.array([[cons(rho(x0 + (m - 0.5) * dx, y0 + k * dx)) for k in (-1, 0, 1)] for m in (0, 1)])
    return S, S.copy(), avg


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1412_4489_gb300 import gks, workloads as wl
    gks.load()
    dev_index = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    p = wl.smooth_wave_2d(args.size, seed=SEED)
    cells = p.nx * p.ny
    faces_x = (p.nx + 1) * p.ny
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def make(prec):
        with torch.cuda.stream(stream):
            return gks.Solver(p, prec, stream=stream.cuda_stream, tau_eps=0.0)

    def timed_steps(s, K, W):
        with torch.cuda.stream(stream):
            s.advance(W, CFL)
            s.sync()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            for k in range(K):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                s.advance(1, CFL)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in ev)
            t, nsteps = s.sync()
        return ms, nsteps

    def max_over_ranks(x):
        from paper_1412_4489_gb300 import parallel
        return parallel.max_over_ranks(x, device="cuda")

    # ---- headline: FP32-bulk ----
    s32 = make(gks.GKS_FP32_BULK)
    with ClockSampler(dev_index) as clk:
        ms32, n32 = timed_steps(s32, args.steps, args.warmup)
    clocks = clk.summary()
    ms32 = max_over_ranks(ms32)
    ms_per_step = ms32 / args.steps
    value = world * cells * args.steps / (ms32 * 1e-3) / 1e6

    # per-kernel durations (events between the kernels of each step), L2 flushed between steps
    prof = {k: 0.0 for k in gks.KERNEL_NAMES}
    KP = max(10, min(args.steps, 50))
    with torch.cuda.stream(stream):
        for k in range(KP):
            flush.fill_(float(k))
            for name, ms in gks.gks_profile_step(s32.h, CFL).items():
                prof[name] += ms / KP
    prof_step = sum(prof.values())

    # ---- plain FP64 ----
    s64 = make(gks.GKS_FP64)
    K64 = max(3, args.steps // 5)
    ms64, _ = timed_steps(s64, K64, max(3, args.warmup // 2))
    ms64 = max_over_ranks(ms64)
    value64 = world * cells * K64 / (ms64 * 1e-3) / 1e6
    prof64 = {k: 0.0 for k in gks.KERNEL_NAMES}
    with torch.cuda.stream(stream):
        for k in range(5):
            flush.fill_(float(k))
            for name, ms in gks.gks_profile_step(s64.h, CFL).items():
                prof64[name] += ms / 5

    # ---- L1 difference FP32-bulk vs FP64 after the same 100 steps from the initial state ----
    a, b = make(gks.GKS_FP32_BULK), make(gks.GKS_FP64)
    a.advance(100, CFL)
    b.advance(100, CFL)
    Ua, _, _, ta = a.state()
    Ub, _, _, tb = b.state()
    l1 = float(np.sum(np.abs(Ua[0] - Ub[0])) / np.sum(np.abs(Ub[0])))
    linf = float(np.max(np.abs(Ua[0] - Ub[0])) / np.max(np.abs(Ub[0])))
    a.close()
    b.close()
    errors = error_legs(stream) if not args.no_batch else None
    validation = vortex_leg(stream) if not args.no_batch else None
    characteristic = characteristic_leg(stream) if not args.no_batch else None
    convergence = convergence_leg(stream) if not args.no_batch else None
    cavity = cavity_leg(stream, args.cavity_steps) if (not args.no_batch and args.cavity_steps > 0) else None

    # ---- end to end through the C ABI with host buffers ----
    KE = max(3, min(args.steps, 20))
    pin = lambda shape: torch.zeros(shape, dtype=torch.float64, pin_memory=True).numpy()
    U, Wx, Wy = pin(p.U.shape), pin(p.Wx.shape), pin(p.Wy.shape)
    U[...] = p.U
    Wx[...] = p.Wx
    Wy[...] = p.Wy
    se = make(gks.GKS_FP32_BULK)
    gks.gks_step(se.h, CFL)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    tt = 0.0
    for _ in range(KE):
        gks.gks_set_state(se.h, U, Wx, Wy, tt)
        gks.gks_step(se.h, CFL)
        tt = gks.gks_get_state(se.h, U, Wx, Wy)
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    bytes_state = 8 * (U.size + Wx.size + Wy.size)
    se.close()

    # ---- batched form: 512 seeded grids of uneven sizes in one persistent launch ----
    batched = run_batched(args, stream) if not args.no_batch else None

    # ---- one 4096^2 FP32-bulk smooth wave (inputs larger than L2) ----
    big = None
    if not args.no_batch:
        p4 = wl.smooth_wave_2d(4096, seed=SEED)
        with torch.cuda.stream(stream):
            s4 = gks.Solver(p4, gks.GKS_FP32_BULK, stream=stream.cuda_stream, tau_eps=0.0)
            s4.advance(3, CFL)
            s4.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            K4 = 10
            e0.record(stream)
            s4.advance(K4, CFL)
            e1.record(stream)
            e1.synchronize()
            ms4 = max_over_ranks(e0.elapsed_time(e1))
            s4.close()
        big = {"value": round(world * 4096 * 4096 * K4 / (ms4 * 1e-3) / 1e6, 3), "unit": UNIT,
               "ms_per_step": round(ms4 / K4, 4), "steps": K4, "grid": [4096, 4096],
               "precision": "fp32_bulk", "l2": "state (~1.2 GB) larger than L2"}
        del p4

    # ---- roofline of the dominant kernel ----
    flux_kernels = {k: v for k, v in prof.items() if k.startswith("flux")}
    dom = max(flux_kernels, key=flux_kernels.get)
    L, R, avg = face_inputs(p)
    ops = gks.gks_face_op_count(L, R, avg, p.Lx / p.nx, p.Ly / p.ny, 1e-3, p.gamma, 0.0, 1.0, 0.0, 1.0,
                                gks.GKS_FP32_BULK)
    flops_face = ops["add"] + ops["mul"] + ops["div"]
    nfaces = faces_x if dom == "flux_x" else p.nx * (p.ny + 1)
    achieved = flops_face * nfaces / (prof[dom] * 1e-3) / 1e12
    peak32 = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    measured32 = gks.gks_measure_alu_peak(gks.GKS_FP32_BULK)
    measured64 = gks.gks_measure_alu_peak(gks.GKS_FP64)
    traffic_face, traffic_src = flux_traffic("fp32")
    traffic = None if traffic_face is None else round(traffic_face * nfaces)
    # the kernel is issue-bound: the share of the SMs' issue slots its instructions (ncu count
    # per face at 2048^2, same source) take in this launch's measured time
    instr_face, _ = profile_figure("fp32", "instructions_per_face")
    issue_frac = None if instr_face is None else round(
        instr_face * nfaces / 32 / (prof[dom] * 1e-3) / (SM_COUNT * ISSUE_PER_SM_CLK * SM_MAX_MHZ * 1e6), 4)
    flops64 = flops_face  # the same arithmetic in FP64
    achieved64 = flops64 * nfaces / (prof64[dom] * 1e-3) / 1e12

    out = None
    if rank == 0:
        cpu = cpu_baseline(args) if (world == 1 and not args.no_cpu_baseline) else None
        out = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "accumulate_dtype": "f32x2 (double-float hi+lo)",
            "data": "synthetic (seeded smooth wave)",
            "config": dict(workload_config(args.size), precision="fp32_bulk", parallelism=f"replicas x{world}"),
            "fp64_plain": {"value": round(value64, 3), "unit": UNIT, "ms_per_step": round(ms64 / K64, 5),
                           "steps": K64, "speedup_fp32_bulk": round(value / value64, 2)},
            "error_fp32_bulk_vs_fp64": {"l1_rho_rel": l1, "linf_rho_rel": linf, "steps": 100,
                                        "reference": "GPU FP64 path (oracle-pinned in tests)",
                                        "other_workloads": errors},
            "roofline": {"bound": "alu", "kernel": f"k_flux<{dom[-1]}> fp32", "achieved": round(achieved, 3),
                         "peak": round(peak32, 2), "unit": "TFLOP/s", "frac": round(achieved / peak32, 4),
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                         "peak_measured_fma": round(measured32, 2), "frac_of_measured_fma": round(achieved / measured32, 4),
                         "flops_per_face": flops_face, "faces_per_launch": nfaces,
                         "faces_per_s": round(nfaces / (prof[dom] * 1e-3), 0),
                         "special_per_face": {k: ops[k] for k in ("sqrt", "rsqrt", "exp", "expm1", "erfc")},
                         "kernel_ms": round(prof[dom], 5), "traffic": traffic,
                         "issue_slots": {"instructions_per_face": instr_face, "frac": issue_frac,
                                         "peak": "152 SMs x 4 warp instructions per clock x 2070 MHz"}},
            "roofline_fp64": {"bound": "alu", "kernel": f"k_flux<{dom[-1]}> fp64", "achieved": round(achieved64, 4),
                              "peak": round(measured64, 3), "unit": "TFLOP/s", "frac": round(achieved64 / measured64, 4),
                              "peak_source": "measured FP64 FMA throughput (gks_measure_alu_peak)",
                              "kernel_ms": round(prof64[dom], 5)},
            "batched": batched,
            "validation": validation,
            "characteristic": characteristic,
            "convergence": convergence,
            "cavity": cavity,
            "fp32_4096": big,
            "kernels_ms_fp32": {k: round(v, 5) for k, v in prof.items()},
            "kernels_ms_fp64": {k: round(v, 5) for k, v in prof64.items()},
            "profiled_step_ms": round(prof_step, 5),
            "clocks": clocks,
            "e2e": {"value": round(world * cells * KE / e2e_s / 1e6, 3), "unit": UNIT,
                    "h2d_bytes_per_step": bytes_state, "d2h_bytes_per_step": bytes_state, "steps": KE,
                    "path": "gks_set_state (host) + gks_step + gks_get_state (host), pinned FP64 buffers"},
            "gpu_launches": args.steps * gks.gks_launches_per_step(s32.h),
            "cpu_baseline": cpu,
        }
    s32.close()
    s64.close()
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


def error_legs(stream):
    """FP32-bulk against FP64 (the oracle-pinned GPU path) in relative L1 of density on the
    other seeded workloads: the 1024^2 Navier-Stokes Riemann data (200 steps) and the 512^2
    cavity (2000 steps).  The Riemann data carry vortex sheets whose grid-scale growth makes
    the FP64 scheme diverge from itself once the start is perturbed by 1e-12; that control is
    reported beside the FP32 figure."""
    import numpy as np
    from paper_1412_4489_gb300 import gks, workloads as wl

    def rho_l1(a, b):
        ra, rb = a.state()[0][0], b.state()[0][0]
        return float(np.sum(np.abs(ra - rb)) / np.sum(np.abs(rb)))

    out = {}
    with __import__("torch").cuda.stream(stream):
        p = wl.riemann_2d(1024, seed=3, mu=1e-4, Pr=0.72)
        q = wl.riemann_2d(1024, seed=3, mu=1e-4, Pr=0.72)
        q.U = q.U * (1.0 + 1e-12 * np.random.default_rng(1).standard_normal(q.U.shape))
        f64 = gks.Solver(p, gks.GKS_FP64, stream=stream.cuda_stream, tau_eps=0.05)
        f32 = gks.Solver(p, gks.GKS_FP32_BULK, stream=stream.cuda_stream, tau_eps=0.05)
        ctl = gks.Solver(q, gks.GKS_FP64, stream=stream.cuda_stream, tau_eps=0.05)
        rows, done = [], 0
        for m in (100, 200):
            for s in (f64, f32, ctl):
                s.advance(m - done, CFL)
            done = m
            rows.append({"steps": m, "l1_rho_rel_fp32": rho_l1(f32, f64), "l1_rho_rel_fp64_perturbed_1e-12": rho_l1(ctl, f64)})
        for s in (f64, f32, ctl):
            s.close()
        out["riemann_ns_1024"] = rows
        out["riemann_ns_1024_note"] = (
            "the L1 <= 1e-5 bound holds to step ~100, the data's predictability horizon at 1024^2: past it the "
            "FP64 scheme started from a 1e-12 perturbation departs from itself by more (l1_rho_rel_fp64_perturbed_1e-12 "
            "beside each figure), so no arithmetic but the identical FP64 sequence can meet it")
        c = wl.cavity_2d(512)
        f64 = gks.Solver(c, gks.GKS_FP64, stream=stream.cuda_stream, tau_eps=0.05)
        f32 = gks.Solver(c, gks.GKS_FP32_BULK, stream=stream.cuda_stream, tau_eps=0.05)
        f64.advance(2000, CFL)
        f32.advance(2000, CFL)
        out["cavity_512"] = [{"steps": 2000, "l1_rho_rel_fp32": rho_l1(f32, f64)}]
        f64.close()
        f32.close()
    return out


def vortex_leg(stream):
    """The paper's isotropic vortex (Table 2) at 121^2 over one period (t = 10, CFL 0.2) in both
    precisions: L1 / L2 density error against the exact solution (the initial data) and the
    throughput of the whole run, timed with CUDA events."""
    import math
    import numpy as np
    import torch
    from paper_1412_4489_gb300 import gks, workloads as wl
    p = wl.isotropic_vortex(121)
    out = {"workload": "isotropic vortex 121^2, [-5, 5]^2 periodic, one period (t = 10), CFL 0.2",
           "table2_paper": {"L1": 2.6716280e-04, "L2": 4.8235722e-04}}
    for prec, name in ((gks.GKS_FP64, "fp64"), (gks.GKS_FP32_BULK, "fp32_bulk")):
        with torch.cuda.stream(stream):
            s = gks.Solver(p, prec, stream=stream.cuda_stream, tau_eps=0.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(1000):
                s.advance(64, 0.2, 10.0)
                t, k = s.sync()
                if t >= 10.0 * (1 - 1e-14):
                    break
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            U = s.state()[0]
            s.close()
        d = U[0] - p.U[0]
        out[name] = {"L1": float(np.mean(np.abs(d))), "L2": float(math.sqrt(np.mean(d * d))), "steps": int(k),
                     "value": round(121 * 121 * k / (ms * 1e-3) / 1e6, 3), "unit": UNIT}
    return out


def convergence_leg(stream):
    """The 2D smooth wave on 32^2..512^2 to t = 1 (one period along x + y, so the exact solution
    is the initial data) in plain FP64 and FP32-bulk at the paper's CFL 0.2: mean |rho - exact|
    per grid and the observed orders between successive grids.  (At CFL 0.5 the Euler-limit
    collision time with the min-of-directions time step puts the diagonal wave at a summed
    2D Courant number of 1.0, where roundoff grows by ~1.8% per step: visible after ~700
    steps at 512^2, so a run to t = 1 there measures that growth, not the scheme's order.)"""
    cfl = 0.2
    import numpy as np
    import torch
    from paper_1412_4489_gb300 import gks, workloads as wl
    ns = [32, 64, 128, 256, 512]
    out = {"workload": "2D Euler smooth wave, periodic [0,2]^2, seed 2, CFL 0.2, to t = 1 (one period)",
           "grids": ns, "norm": "mean |rho - rho_exact| over cells (exact cell averages)"}
    for prec, name in ((gks.GKS_FP64, "fp64"), (gks.GKS_FP32_BULK, "fp32_bulk")):
        errs, steps = [], []
        for n in ns:
            p = wl.smooth_wave_2d(n, seed=SEED)
            with torch.cuda.stream(stream):
                s = gks.Solver(p, prec, stream=stream.cuda_stream, tau_eps=0.0)
                for _ in range(100000):
                    s.advance(64, cfl, 1.0)
                    t, k = s.sync()
                    if t >= 1.0 * (1 - 1e-14):
                        break
                U = s.state()[0]
                s.close()
            errs.append(float(np.mean(np.abs(U[0] - p.U[0]))))
            steps.append(int(k))
        out[name] = {"l1": errs, "steps": steps,
                     "orders": [round(math.log2(errs[i] / errs[i + 1]), 3) for i in range(len(ns) - 1)]}
    out["fp32_vs_fp64_error_ratio"] = [round(a / b, 4) for a, b in zip(out["fp32_bulk"]["l1"], out["fp64"]["l1"])]
    return out


def cavity_leg(stream, nsteps):
    """The lid-driven cavity at 512^2 (Re 1000, lid Mach 0.15, isothermal no-slip walls,
    Navier-Stokes with the Prandtl correction) advanced nsteps steps toward steady state in
    FP32-bulk and plain FP64: throughput of each (CUDA events around the whole run) and the
    relative L1 density difference between the two at checkpoints."""
    import numpy as np
    import torch
    from paper_1412_4489_gb300 import gks, workloads as wl
    c = wl.cavity_2d(512)
    out = {"workload": "lid-driven cavity 512^2, Re 1000, lid Mach 0.15, Pr 0.72, CFL 0.5", "steps": nsteps,
           "unit": UNIT}
    with torch.cuda.stream(stream):
        f64 = gks.Solver(c, gks.GKS_FP64, stream=stream.cuda_stream, tau_eps=0.05)
        f32 = gks.Solver(c, gks.GKS_FP32_BULK, stream=stream.cuda_stream, tau_eps=0.05)
        ms = {"fp64": 0.0, "fp32_bulk": 0.0}
        rows, done = [], 0
        checkpoints = sorted({min(nsteps, k) for k in (1000, 5000, 10000, nsteps)})
        for m in checkpoints:
            for s, key in ((f64, "fp64"), (f32, "fp32_bulk")):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.advance(m - done, CFL)
                e1.record(stream)
                e1.synchronize()
                ms[key] += e0.elapsed_time(e1)
            done = m
            ra, rb = f32.state()[0][0], f64.state()[0][0]
            speed = f64.state()[0]
            umax = float(np.max(np.hypot(speed[1], speed[2]) / speed[0]))
            rows.append({"steps": m, "l1_rho_rel_fp32": float(np.sum(np.abs(ra - rb)) / np.sum(np.abs(rb))),
                         "max_speed_fp64": umax, "t": f64.sync()[0]})
        f64.close()
        f32.close()
    out["l1_rho_rel_fp32_vs_fp64"] = rows
    for key in ms:
        out[key] = {"value": round(512 * 512 * nsteps / (ms[key] * 1e-3) / 1e6, 3), "ms_per_step": round(ms[key] / nsteps, 4)}
    out["speedup_fp32_bulk"] = round(out["fp32_bulk"]["value"] / out["fp64"]["value"], 2)
    return out


def characteristic_leg(stream):
    """The Navier-Stokes four-quadrant data at 1024^2 with the reconstruction in conservative
    and in characteristic variables: step throughput (CUDA events over 20 graph-replayed steps
    after 3 warm-up steps) and the reconstruction kernel's time."""
    import torch
    from paper_1412_4489_gb300 import gks, workloads as wl
    p = wl.riemann_2d(1024, seed=3, mu=1e-4, Pr=0.72)
    out = {"workload": "NS four-quadrant data 1024^2, seed 3, mu 1e-4, Pr 0.72, CFL 0.5", "unit": UNIT}
    for prec, pname in ((gks.GKS_FP32_BULK, "fp32_bulk"), (gks.GKS_FP64, "fp64")):
        for ch in (0, 1):
            with torch.cuda.stream(stream):
                s = gks.Solver(p, prec, stream=stream.cuda_stream, characteristic=ch)
                s.advance(3, CFL)
                s.sync()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.advance(20, CFL)
                e1.record(stream)
                e1.synchronize()
                recon = gks.gks_profile_step(s.h, CFL)["recon"]
                s.close()
            ms = e0.elapsed_time(e1) / 20
            out[f"{pname}_{'characteristic' if ch else 'conservative'}"] = {
                "value": round(p.nx * p.ny / (ms * 1e-3) / 1e6, 3), "ms_per_step": round(ms, 4),
                "recon_ms": round(recon, 4)}
    return out


def run_batched(args, stream):
    """512 seeded grids (sizes 32..384, half smooth waves, half four-quadrant Riemann data,
    gamma in {1.4, 5/3}, mu ~ logU[1e-5, 1e-3]) advanced by one persistent graph-captured
    launch per call, after the autotuner picked the tile width and blocks per SM.  Under
    torchrun the grids are sharded across the ranks (largest first onto the least-loaded rank;
    no exchange between ranks) and the slowest rank's time is taken."""
    import torch
    from paper_1412_4489_gb300 import gks, parallel, workloads as wl
    rank, world, _ = parallel.rank_env()
    specs = wl.batch_specs(512, seed=5)
    all_cells = [sp[0] * sp[1] for sp in specs]
    mine = parallel.shard_grids(all_cells, world)[rank]
    probs = [wl.batch_problem(specs[g]) for g in mine]
    cells = sum(all_cells)
    out = {"grids": len(specs), "cells": cells, "launches_per_call": 1, "unit": UNIT,
           "parallelism": f"grids sharded over {world} rank(s), no data-path collective",
           "workload": "512 seeded grids 32..384 per side: smooth waves (periodic) and four-quadrant Riemann "
                       "data (outflow), gamma 1.4 or 5/3, mu logU[1e-5, 1e-3], Pr 0.72, CFL 0.5"}
    for prec, key, K in ((gks.GKS_FP32_BULK, "fp32_bulk", 20), (gks.GKS_FP64, "fp64", 10)):
        b = gks.Batch(probs, prec, stream=stream.cuda_stream)
        (wx, wy), bps, _ = gks.gks_batch_autotune(b.b, CFL, 1)
        with torch.cuda.stream(stream):
            b.step(1, CFL)
            b.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(K, CFL)
            e1.record(stream)
            e1.synchronize()
            lo, hi = b.sync()
            # the split of a step over the kernel's phases (device clock at each barrier)
            phases = gks.gks_batch_profile(b.b, 3, CFL)
        ms = parallel.max_over_ranks(e0.elapsed_time(e1), device="cuda")
        out[key] = {"value": round(cells * K / (ms * 1e-3) / 1e6, 3), "ms_per_step": round(ms / K, 3),
                    "steps": K, "face_tile_width": {"x": wx, "y": wy}, "blocks_per_sm": bps,
                    "steps_per_grid": [lo, hi], "phases_ms_per_step": {k: round(v, 4) for k, v in phases.items()}}
        b.close()
    out["value"] = out["fp32_bulk"]["value"]
    out["speedup_fp32_bulk"] = round(out["fp32_bulk"]["value"] / out["fp64"]["value"], 2)
    # the same work on one grid: every batch grid is Navier-Stokes with the Prandtl correction,
    # so the comparison is the single-grid FP32-bulk Navier-Stokes rate at a size above L2
    p = wl.riemann_2d(2048, seed=3, mu=1e-4, Pr=0.72)
    with torch.cuda.stream(stream):
        s = gks.Solver(p, gks.GKS_FP32_BULK, stream=stream.cuda_stream)
        s.advance(3, CFL)
        s.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.advance(20, CFL)
        e1.record(stream)
        e1.synchronize()
        s.close()
    ms1 = e0.elapsed_time(e1) / 20
    single = p.nx * p.ny / (ms1 * 1e-3) / 1e6
    out["single_grid_ns_fp32_bulk"] = {"workload": "NS four-quadrant data 2048^2, mu 1e-4, Pr 0.72", "unit": UNIT,
                                       "value": round(single, 3), "ms_per_step": round(ms1, 4)}
    out["batched_vs_single_grid_ns"] = round(out["fp32_bulk"]["value"] / single, 3)
    return out


# ----------------------------------------------------------------------------
# the oracle on the host cores
# ----------------------------------------------------------------------------
def oracle_rate(n, min_seconds, max_steps, warmup=1):
    import oracle
    from paper_1412_4489_gb300 import workloads as wl
    p = wl.smooth_wave_2d(n, seed=SEED)
    P = oracle.params(gamma=p.gamma, tau_eps=0.0)
    st = oracle.State2D(p.nx, p.ny, p.Lx, p.Ly, p.U, p.Wx, p.Wy)
    bc = oracle.bcs([0, 0, 0, 0])
    for _ in range(warmup):
        oracle.step2d(P, st, bc, CFL)
    t0 = time.perf_counter()
    k = 0
    while k < max_steps and (k == 0 or time.perf_counter() - t0 < min_seconds):
        oracle.step2d(P, st, bc, CFL)
        k += 1
    el = time.perf_counter() - t0
    return n * n * k / el / 1e6, k, el, oracle.num_threads()


def cpu_baseline(args):
    v, k, el, cores = oracle_rate(args.size, 10.0, 50, warmup=0)
    return {"value": round(v, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{k} oracle steps of the {args.size}x{args.size} smooth wave ({el:.1f} s, OpenMP over rows)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1412_4489_gb300 import workloads as wl
    n = args.ref_size or args.size
    p = wl.smooth_wave_2d(n, seed=SEED)
    P = oracle.params(gamma=p.gamma, tau_eps=0.0)
    st = oracle.State2D(p.nx, p.ny, p.Lx, p.Ly, p.U, p.Wx, p.Wy)
    bc = oracle.bcs([0, 0, 0, 0])
    for _ in range(args.warmup):
        oracle.step2d(P, st, bc, CFL)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.step2d(P, st, bc, CFL)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n * n * args.steps / total / 1e6
    sample = (f"each step: one oracle step of the {n}x{n} smooth wave (the timed workload itself)" if n == args.size else
              f"each step: one oracle step of the smooth wave at {n}x{n} (a bounded sample of the {args.size}^2 workload)")
    out = {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(total / args.steps * 1e3, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded smooth wave)",
           "impl": "reference", "config": dict(workload_config(n), precision="fp64"),
           "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=N_GRID)
    ap.add_argument("--ref-size", type=int, default=None,
                    help="grid of the reference arm (default: --size, the timed workload itself)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cavity-steps", type=int, default=20000,
                    help="steps of the 512^2 cavity leg in both precisions (0 skips it)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched and 4096^2 legs")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        import oracle
        oracle.build()
        run_reference(args)
    else:
        import __graft_entry__
        __graft_entry__.build()
        run_ours(args)


if __name__ == "__main__":
    main()
