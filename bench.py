#!/usr/bin/env python
"""Benchmark of the fused TVD-RK3 level-set step (LevelSetPy, arXiv 2507.11542) on GB300.

Workload: the air3D pursuit-evasion game on a 101^3 grid over
[-6,20]x[-10,10]x[0,2pi) (psi periodic), va = vb = 5, |a|,|b| <= 1,
V0 = sqrt(x^2+y^2) - 5, WENO5 + Lax-Friedrichs + TVD-RK3, CFL 0.8, BRT
min(0, H). One step = one full RK3 step (one hj_rk3_step call: three fused stage
kernels) over the whole grid; the metric is cell-updates/s (one node advanced
one RK3 step).

  value  : FP64 (the paper's precision) device-resident throughput, L2 flushed
           between timed steps; roofline against the measured DFMA ceiling
  fp32   : the same in FP32, with its error against the FP64 solve over the
           whole horizon; roofline against the measured FFMA ceiling
  e2e    : FP64 hj_solve through the C ABI with pinned host buffers: V0
           uploaded, the first time slice (tau = 0.28) integrated, V
           downloaded, per step
  batched / served : the 64-instance mix in one batched solve; Poisson-arriving
           requests through the server; FP32 with each result's error against
           FP64 stated
  large_grids : the expanding sphere on 512^3 (FP32: WENO5, ENO1, ENO2) and the
           Dubins car on 81^4 (FP32, FP64), device-resident steps, with their
           HBM fraction
  cpu_baseline / --impl reference : the FP64 CPU oracle on the host cores

Run: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
(N > 1 under torch.distributed.run: independent replicas, one per GPU.)
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CELLS = 101 ** 3
HORIZON = 2.8
E2E_TAU = 0.28
# Algorithmic work of one fused stage launch per node (air3D, WENO5), derived
# operation by operation in the design notes: FP ops (an FMA counts 2) and
# HBM words (stage 1 reads V and writes V1: 2 words; stages 2 and 3 read the
# stage input and V^n and write one array: 3 words).
FLOPS_PER_NODE_STAGE = 475
WORDS_PER_NODE_STEP = 8
# DRAM bytes (read + write) of one stage-2 launch of the row kernel on this
# workload, from the ncu captures of the kernel as it stands (the 101^3 arrays
# stay in L2, so DRAM traffic is below the algorithmic bytes); None where the
# kernel changed after the capture.
NCU_TRAFFIC_BYTES = {"float64": 16.57e6, "float32": 8.29e6}
# FP32 / FP64 lanes per SM on GB300 (FMA = 2 flops): the unit-count peak given
# beside the measured one
LANES_PER_SM = {"float32": 128, "float64": 2}
SM_MAX_MHZ = 2070.0
L2_FLUSH_BYTES = 256 << 20


def sm_count(device: int = 0) -> int:
    import torch
    return int(torch.cuda.get_device_properties(device).multi_processor_count)


def alu_peaks(device: int):
    """Measured FFMA and DFMA ceilings of this GPU (TFLOP/s): the best of five
    launches of the FMA-throughput probe (libhj_peak.so), beside the peaks
    from unit counts at the maximum SM clock."""
    import ctypes
    from paper_2507_11542_gb300 import build
    lib = ctypes.CDLL(build.build_peak())
    lib.hj_alu_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double)]
    out = {}
    sms = sm_count(device)
    for name, code in (("float32", 1), ("float64", 2)):
        tf, ms = ctypes.c_double(0), ctypes.c_double(0)
        rc = lib.hj_alu_peak(device, code, 5, ctypes.byref(tf), ctypes.byref(ms))
        if rc != 0:
            raise RuntimeError("FMA-throughput probe failed (%d)" % rc)
        out[name] = {"measured_tflops": tf.value, "probe_ms": ms.value,
                     "unit_count_tflops": sms * LANES_PER_SM[name] * 2 * SM_MAX_MHZ * 1e6 / 1e12,
                     "unit_count_source": "%d SMs x %d lanes x 2 flops x %.0f MHz"
                                          % (sms, LANES_PER_SM[name], SM_MAX_MHZ)}
    return out


def measured_hbm_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
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

    def __exit__(self, *exc):
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
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(items, rank: int, world: int):
    """The share of independent instances one rank solves: every world-th item
    starting at its rank (no data crosses ranks)."""
    return items[rank::world]


def job_rate(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job throughput from each rank's units and its own time: all
    ranks' units divided by the slowest rank's time (weak scaling)."""
    slowest = max_over_ranks(seconds, world)
    return sum_over_ranks(units_per_rank, world) / slowest


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def workload():
    from paper_2507_11542_gb300 import workloads as W
    spec, V0 = W.air3d(101)
    return spec, V0


def run_steps(ctx, spec, m, V, bufs, dt, K, flush, events, per_stage=False):
    """K RK3 steps with an L2 flush before every step: one hj_rk3_step call per
    step (the library's step entry point: its three fused stage kernels), or,
    with per_stage, three hj_rk3_stage calls with an event between stages.
    Returns per-step and (per_stage) per-stage-launch durations in ms."""
    import ctypes
    import torch
    from paper_2507_11542_gb300 import _lib
    u1, u2 = bufs
    lib = _lib.load()
    g = ctypes.byref(_lib.make_grid(spec))
    mm = ctypes.byref(m)
    code = _lib.dtype_code(V.dtype)
    h, pv, p1, p2 = ctypes.c_void_p(ctx.handle), ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(u1.data_ptr()), \
        ctypes.c_void_p(u2.data_ptr())
    calls = [(1, pv, None, p1), (2, p1, pv, p2), (3, p2, pv, pv)]
    step_ms, stage_ms = [], []
    for k in range(K):
        if flush is not None:
            flush.zero_()
        ev = events[k] if events is not None else None
        if ev:
            ev[0].record()
        if per_stage:
            for s, (stage, u, vn, out) in enumerate(calls):
                st = lib.hj_rk3_stage(h, g, mm, code, stage, u, vn, out, dt)
                if st != 0:
                    raise _lib.HJError(st, _lib.hj_ctx_last_error(ctx.handle))
                if ev:
                    ev[s + 1].record()
        else:
            st = lib.hj_rk3_step(h, g, mm, code, pv, dt)
            if st != 0:
                raise _lib.HJError(st, _lib.hj_ctx_last_error(ctx.handle))
            if ev:
                ev[3].record()
    torch.cuda.synchronize()
    if events is not None:
        for k in range(K):
            ev = events[k]
            step_ms.append(ev[0].elapsed_time(ev[3]))
            if per_stage:
                stage_ms.extend([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])])
    return step_ms, stage_ms


def bench_dtype(ctx, spec, V0, dtype, K, W_, world, flush, m=None):
    """Timed: K steps through hj_rk3_step (the metric). Then K steps through
    hj_rk3_stage with events between the stages, for the per-launch duration
    of the stage kernel (the roofline)."""
    import torch
    from paper_2507_11542_gb300 import solver
    if m is None:
        m = solver.method(dynamics=2, params=(5.0, 5.0, 1.0, 1.0), brt=1)
    sbi = solver.step_bound(ctx, spec, m)
    dt = 0.8 / sbi
    tdt = getattr(torch, dtype)
    V = torch.from_numpy(np.ascontiguousarray(V0.ravel(order="F"))).to("cuda", tdt)
    u1, u2 = torch.empty_like(V), torch.empty_like(V)
    run_steps(ctx, spec, m, V, (u1, u2), dt, W_, flush, None)
    run_steps(ctx, spec, m, V, (u1, u2), dt, W_, flush, None, per_stage=True)
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    barrier(world)
    torch.cuda.synchronize()
    step_ms, _ = run_steps(ctx, spec, m, V, (u1, u2), dt, K, flush, events)
    torch.cuda.synchronize()
    barrier(world)
    _, stage_ms = run_steps(ctx, spec, m, V, (u1, u2), dt, K, flush, events, per_stage=True)
    assert torch.isfinite(V).all().item()
    total_ms = max_over_ranks(sum(step_ms), world)
    return {"total_ms": total_ms, "ms_per_step": total_ms / K, "stage_ms": stage_ms,
            "launch_ms_mean": sum(stage_ms) / len(stage_ms), "launches": 3 * K, "dt": dt}


def bench_e2e(ctx, spec, V0, dtype, K, W_, world):
    """hj_solve with pinned host input/output: H2D of V0, the steps to tau = 0.28, D2H of V."""
    import torch
    from paper_2507_11542_gb300 import solver
    m = solver.method(dynamics=2, params=(5.0, 5.0, 1.0, 1.0), brt=1)
    tdt = getattr(torch, dtype)
    v0 = torch.from_numpy(np.ascontiguousarray(V0.ravel(order="F"))).to(tdt).pin_memory()
    out = torch.empty((1, v0.numel()), dtype=tdt).pin_memory()
    for _ in range(W_):
        solver.solve(ctx, spec, m, v0, [E2E_TAU], out=out)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps = launches = 0
    for _ in range(K):
        _, _, st = solver.solve(ctx, spec, m, v0, [E2E_TAU], out=out)
        steps += st["steps"]
        launches += st["kernel_launches"]
    torch.cuda.synchronize()
    el = max_over_ranks(time.perf_counter() - t0, world)
    return {"value": world * steps * N_CELLS / el, "unit": "cell-updates/s",
            "h2d_bytes_per_step": int(v0.numel() * v0.element_size()),
            "d2h_bytes_per_step": int(out.numel() * out.element_size()),
            "rk3_steps_per_step": steps // K, "launches": launches}


def bench_surface(ctx, hbm, reps=20):
    """hj_implicit_surface on the 512^3 grid (FP32): the union of two spheres
    written to HBM; bytes written = 4 per node."""
    import torch
    from paper_2507_11542_gb300 import solver, workloads as W
    spec, _ = W.expanding_sphere(512)
    shapes = [{"kind": 1, "center": (-0.3, 0.0, 0.0), "radius": 0.25},
              {"kind": 1, "op": 1, "center": (0.3, 0.1, 0.0), "radius": 0.2}]
    n = int(np.prod(spec.n))
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    for _ in range(3):
        solver.implicit_surface(ctx, spec, shapes, out=out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        solver.implicit_surface(ctx, spec, shapes, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    gbs = 4 * n / (ms / 1e3) / 1e9
    return {"ms": ms, "cells": n, "hbm_achieved_gbs": gbs, "hbm_frac": gbs / hbm, "bound": "hbm",
            "what": "initial surface (union of two spheres) written by the device, FP32"}


def bench_rockets(ctx):
    """The paper's rockets game as it runs it: 100^3 over [-64, 64], 11 slices
    over a 2.5 s horizon, BRT with the positive rule; one hj_solve with host
    input and output (V0 up, 11 slices down), FP64 ENO2 as the paper, and
    FP32 WENO5."""
    import torch
    from paper_2507_11542_gb300 import solver, workloads as W
    spec, V0 = W.rockets(100)
    ts = list(W.slice_times(2.5))
    out = {}
    for name, dtype, scheme in (("fp64_eno2", "float64", 2), ("fp32_weno5", "float32", 5)):
        m = solver.method(scheme=scheme, dynamics=7, params=(1.0, 32.0, 1.0, 1.0), brt=1)
        tdt = getattr(torch, dtype)
        v0 = torch.from_numpy(np.ascontiguousarray(V0.ravel(order="F"))).to(tdt).pin_memory()
        res = torch.empty((len(ts), v0.numel()), dtype=tdt).pin_memory()
        solver.solve(ctx, spec, m, v0, ts[:2], out=res[:2])  # warm-up (tuning, tables)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, st = solver.solve(ctx, spec, m, v0, ts, out=res)
        el = time.perf_counter() - t0
        out[name] = {"seconds": el, "steps": st["steps"], "cell_updates_per_s": st["cell_updates"] / el}
    out["context"] = ("the paper's Table 1: 11.52 s (global) on a Quadro RTX 4000 with CuPy in FP64, "
                      "ENO2; another machine, quoted as context")
    return out


def bench_large(ctx, world, flush, only=None):
    """The grids far larger than L2: the expanding sphere on 512^3 (FP32) and
    the Dubins car on 81^4 (FP32 and FP64), device-resident RK3 steps. Their
    HBM fraction counts the algorithmic 8 words per cell-update. only: the
    names of the cases to run (None: all, with the initial-surface kernel)."""
    from paper_2507_11542_gb300 import solver, workloads as W
    hbm, _ = measured_hbm_gbs()
    out = {}
    sphere = W.expanding_sphere(512)
    cases = [("sphere512_f32", sphere, solver.method(dynamics=4, params=(1.0,), brt=0), "float32", 10),
             ("sphere512_f32_eno1", sphere, solver.method(scheme=1, dynamics=4, params=(1.0,), brt=0), "float32", 10),
             ("sphere512_f32_eno2", sphere, solver.method(scheme=2, dynamics=4, params=(1.0,), brt=0), "float32", 10),
             ("dubins81_f32", W.dubins4d(81), solver.method(dynamics=3, params=(1.0, 0.5), brt=1), "float32", 6),
             ("dubins81_f64", W.dubins4d(81), solver.method(dynamics=3, params=(1.0, 0.5), brt=1), "float64", 3)]
    if only is None:
        out["surface512_f32"] = bench_surface(ctx, hbm)
    for name, (spec, V0), m, dtype, K in cases:
        if only is not None and name not in only:
            continue
        n = int(np.prod(spec.n))
        r = bench_dtype(ctx, spec, V0, dtype, K, 3, world, flush, m=m)
        rate = world * n / (r["ms_per_step"] / 1e3)
        gbs = 8 * (4 if dtype == "float32" else 8) * n / (r["ms_per_step"] / 1e3) / 1e9
        out[name] = {"value": rate, "unit": "cell-updates/s", "ms_per_step": r["ms_per_step"], "steps": K,
                     "cells": n, "hbm_achieved_gbs": gbs, "hbm_frac": gbs / hbm,
                     "stage_launch_ms_mean": r["launch_ms_mean"]}
    return out


def _mix_problems(mix, dtype):
    import torch
    from paper_2507_11542_gb300 import solver
    specs, methods, v0s, tss = [], [], [], []
    for kind, g, V0, horizon in mix:
        specs.append(g)
        if kind == "di":
            methods.append(solver.method(dynamics=1, params=(1.0,), brt=1))
        elif kind == "air3d":
            methods.append(solver.method(dynamics=2, params=(5.0, 5.0, 1.0, 1.0), brt=1))
        else:
            methods.append(solver.method(dynamics=3, params=(1.0, 0.5), brt=1))
        v0s.append(torch.from_numpy(np.ascontiguousarray(V0.ravel(order="F"))).to("cuda", getattr(torch, dtype)))
        tss.append([0.0, horizon])
    return specs, methods, v0s, tss


def bench_batch(ctx, fp64_subset: int = 8, rank: int = 0, world: int = 1):
    """The 64-instance batched workload (seed 42): FP32 hj_solve_batch, the same
    instances one by one with hj_solve (FP32), and FP64 one by one on a subset.
    With several ranks each solves its shard of the 64 instances."""
    import torch
    from paper_2507_11542_gb300 import solver, workloads as W
    mix = shard(W.batch_mix(42), rank, world)
    specs, methods, v0s, tss = _mix_problems(mix, "float32")
    solver.solve_batch(ctx, specs, methods, v0s, tss)  # warm-up: launch shapes are tuned once
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    outs, times, stats = solver.solve_batch(ctx, specs, methods, v0s, tss)
    torch.cuda.synchronize()
    el_batch = time.perf_counter() - t0
    cells = sum(st["cell_updates"] for st in stats)
    rate = job_rate(cells, el_batch, world)
    launches = stats[0]["kernel_launches"]
    t0 = time.perf_counter()
    for g, m, v, ts in zip(specs, methods, v0s, tss):
        solver.solve(ctx, g, m, v, ts)
    torch.cuda.synchronize()
    el_serial = time.perf_counter() - t0
    sub = list(range(0, len(mix), max(1, len(mix) // fp64_subset)))[:fp64_subset]
    s64, m64, v64, t64 = _mix_problems([mix[i] for i in sub], "float64")
    cells64 = 0
    t0 = time.perf_counter()
    for g, m, v, ts in zip(s64, m64, v64, t64):
        _, _, st = solver.solve(ctx, g, m, v, ts)
        cells64 += st["cell_updates"]
    torch.cuda.synchronize()
    el64 = time.perf_counter() - t0
    # each FP32 result against the same instance solved in FP64 (one batched FP64 solve)
    a64, am64, av64, at64 = _mix_problems(mix, "float64")
    ref, _, _ = solver.solve_batch(ctx, a64, am64, av64, at64)
    errs = [fp32_instance_error(outs[k][-1], ref[k][-1], specs[k], "%s %s" % (mix[k][0], "x".join(map(str, specs[k].n))))
            for k in range(len(mix))]
    return {"workload": "64 solves: 32 double integrator n~U{51..201}, 32 air3D n~U{41..121}, seed 42, FP32"
                        + (", sharded over %d ranks" % world if world > 1 else ""),
            "value": rate, "unit": "cell-updates/s", "seconds": el_batch, "kernel_launches": launches,
            "serial_fp32": cells / el_serial, "serial_fp64": cells64 / el64,
            "serial_fp64_sample": "%d of the 64 instances, one hj_solve each" % len(sub),
            "fp32_error": error_summary(errs, "every instance at its horizon, FP32 against its FP64 solve")}


def fp32_instance_error(a, b, spec, name):
    """One FP32 result against the FP64 solve of the same problem: max|dV| /
    max|V| and the zero-level-set displacement in cells (edge crossings), and
    whether the FP64 zero set meets an extrapolated edge (where the R3 ghost
    rule's sign(v0) can differ between precisions)."""
    A = a.double().cpu().numpy().reshape(spec.n, order="F")
    B = b.double().cpu().numpy().reshape(spec.n, order="F")
    return {"instance": name, "max_abs_err_rel": float(np.max(np.abs(A - B)) / max(np.max(np.abs(B)), 1e-300)),
            "zero_set_displacement_cells": zero_set_displacement_cells(A, B),
            "zero_set_meets_extrapolated_edge": meets_extrapolated_edge(B, spec)}


def meets_extrapolated_edge(V, spec) -> bool:
    for d in range(V.ndim):
        if d in spec.periodic:
            continue
        for idx in (0, V.shape[d] - 1):
            face = np.take(V, idx, axis=d)
            if (face > 0).any() and (face <= 0).any():
                return True
    return False


def error_summary(errs, what):
    cells = [e["zero_set_displacement_cells"] for e in errs]
    over = [e for e in errs if e["zero_set_displacement_cells"] >= 0.1]
    return {"what": what, "instances": len(errs), "bar_cells": 0.1,
            "zero_set_displacement_cells_max": max(cells), "zero_set_displacement_cells_median": float(np.median(cells)),
            "max_abs_err_rel_max": max(e["max_abs_err_rel"] for e in errs),
            "over_bar": len(over),
            "over_bar_instances": [{"instance": e["instance"], "cells": e["zero_set_displacement_cells"],
                                    "reason": ("zero set meets an extrapolated edge: the away-from-zero ghost rule "
                                               "takes sign(v0) at the edge node, which FP32 and FP64 can disagree on"
                                               if e["zero_set_meets_extrapolated_edge"] else "none identified")}
                                   for e in over]}


def bench_serve(ctx, n_req: int, seed: int = 7, load: float = 0.8, budget_gb: float = 64.0, err_samples: int = 16):
    """Poisson arrivals of reachability requests (types uniform over double
    integrator, air3D, Dubins4D; 2-D n~U{51..301}, 3-D n~U{41..161}, 4-D
    n~U{31..81}; horizon ~U[0.5, 3]; FP32) at `load` times the capacity
    measured by serving the same requests all at once."""
    import torch
    from paper_2507_11542_gb300 import solver, workloads as W
    rng = np.random.default_rng(seed)
    mix = []
    for _ in range(n_req):
        kind = int(rng.integers(0, 3))
        horizon = float(rng.uniform(0.5, 3.0))
        if kind == 0:
            g, V0 = W.double_integrator(int(rng.integers(51, 302)), float(rng.uniform(0.2, 0.8)))
            mix.append(("di", g, V0, horizon))
        elif kind == 1:
            g, V0 = W.air3d(int(rng.integers(41, 162)), float(rng.uniform(3.0, 7.0)))
            mix.append(("air3d", g, V0, horizon))
        else:
            g, V0 = W.dubins4d(int(rng.integers(31, 82)), seed=int(rng.integers(0, 1 << 30)))
            mix.append(("dubins", g, V0, horizon))
    specs, methods, v0s, tss = _mix_problems(mix, "float32")
    budget = int(budget_gb * (1 << 30))
    with solver.Server(ctx, hbm_budget=budget, max_slots=64) as srv:
        # capacity: everything submitted at once
        t0 = time.perf_counter()
        tickets = [srv.submit(g, m, v, ts) for g, m, v, ts in zip(specs, methods, v0s, tss)]
        for t in tickets:
            srv.wait(t)
        cap_s = time.perf_counter() - t0
        rate = load * n_req / cap_s
        gaps = rng.exponential(1.0 / rate, size=n_req)
        lat, cells = [], 0
        t0 = time.perf_counter()
        tickets = []
        next_t = t0
        for k in range(n_req):
            next_t += gaps[k]
            while time.perf_counter() < next_t:
                time.sleep(min(0.001, max(0.0, next_t - time.perf_counter())))
            tickets.append(srv.submit(specs[k], methods[k], v0s[k], tss[k]))
        sampled = set(range(0, n_req, max(1, n_req // err_samples)))
        kept = {}
        queued = []
        for k, t in enumerate(tickets):
            st, out, times, stats = srv.wait(t)
            lat.append(stats["elapsed_ms"])
            queued.append(stats["queued_ms"])
            cells += stats["cell_updates"]
            if k in sampled:
                kept[k] = out[-1]
        el = time.perf_counter() - t0
        launches = srv.counters()["kernel_launches"]
    lat, queued = np.array(lat), np.array(queued)
    kinds = np.array([m[0] for m in mix])
    by_class = {}
    for kind, label in (("di", "2-D double integrator"), ("air3d", "3-D air3D"), ("dubins", "4-D Dubins car")):
        sel = kinds == kind
        if sel.any():
            by_class[label] = {"requests": int(sel.sum()), "p50_ms": float(np.percentile(lat[sel], 50)),
                               "p99_ms": float(np.percentile(lat[sel], 99)),
                               "queued_p50_ms": float(np.percentile(queued[sel], 50)),
                               "queued_p99_ms": float(np.percentile(queued[sel], 99))}
    worst = np.argsort(lat)[-max(1, n_req // 100):]   # the requests at or above p99
    # sampled results against the same requests solved in FP64 (one batched FP64 solve)
    ks = sorted(kept)
    s64, m64, v64, t64 = _mix_problems([mix[k] for k in ks], "float64")
    ref, _, _ = solver.solve_batch(ctx, s64, m64, v64, t64)
    errs = [fp32_instance_error(kept[k], ref[i][-1], specs[k], "request %d (%s %s)" % (k, mix[k][0],
                                                                                    "x".join(map(str, specs[k].n))))
            for i, k in enumerate(ks)]
    return {"workload": "%d requests, seed %d, Poisson arrivals at %.2f req/s (%.1fx of capacity %.2f req/s), FP32, "
                        "HBM budget %.0f GB" % (n_req, seed, rate, load, n_req / cap_s, budget_gb),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "value": cells / el, "unit": "cell-updates/s", "capacity_req_per_s": n_req / cap_s,
            "kernel_launches": launches,
            "latency_split": {"queued_p50_ms": float(np.percentile(queued, 50)),
                              "queued_p99_ms": float(np.percentile(queued, 99)),
                              "on_device_p50_ms": float(np.percentile(lat - queued, 50)),
                              "on_device_p99_ms": float(np.percentile(lat - queued, 99)),
                              "what": "queued: submission to admission; on device: admission to retirement"},
            "by_class": by_class,
            "slowest_1pct": {"classes": {str(c): int(np.sum(kinds[worst] == c)) for c in set(kinds[worst])},
                             "queued_ms_median": float(np.median(queued[worst])),
                             "latency_ms_median": float(np.median(lat[worst]))},
            "fp32_error": error_summary(errs, "%d sampled requests (every %d-th), FP32 against the same request "
                                              "solved in FP64" % (len(ks), max(1, n_req // err_samples)))}


def zero_set_displacement_cells(V, Vref):
    """Zero-level-set displacement in cells, measured on grid edges: where both
    fields change sign along an edge, |s - s_ref| of the linearly interpolated
    crossing points; where only one does, the distance from that crossing to
    the nearer end of the edge (a lower bound of the move). Max over edges."""
    worst = 0.0
    pos, pos_r = V > 0, Vref > 0
    for d in range(V.ndim):
        a = [slice(None)] * V.ndim
        b = [slice(None)] * V.ndim
        a[d], b[d] = slice(0, V.shape[d] - 1), slice(1, V.shape[d])
        a, b = tuple(a), tuple(b)
        c, cr = pos[a] != pos[b], pos_r[a] != pos_r[b]
        with np.errstate(divide="ignore", invalid="ignore"):
            s = np.nan_to_num(V[a] / (V[a] - V[b]))
            sr = np.nan_to_num(Vref[a] / (Vref[a] - Vref[b]))
        both, only = c & cr, c ^ cr
        if both.any():
            worst = max(worst, float(np.max(np.abs(s - sr)[both])))
        if only.any():
            t = np.where(c, s, sr)[only]
            worst = max(worst, float(np.max(np.minimum(t, 1.0 - t))))
    return worst


def bench_fp32_error(ctx, spec, V0):
    """The FP32 path's error on the bench workload over its whole horizon: the
    11 slices to tau = 2.8 in FP32 against the same solve in FP64 (which the
    parity tests hold within 1e-12 of the oracle)."""
    import torch
    from paper_2507_11542_gb300 import solver, workloads as W
    m = solver.method(dynamics=2, params=(5.0, 5.0, 1.0, 1.0), brt=1)
    ts = W.slice_times(2.8)
    flat = torch.from_numpy(np.ascontiguousarray(V0.ravel(order="F"))).cuda()
    s32, _, st = solver.solve(ctx, spec, m, flat.float(), ts)
    s64, _, _ = solver.solve(ctx, spec, m, flat.double(), ts)
    worst_rel, worst_cells = 0.0, 0.0
    for k in range(1, len(ts)):
        a = s32[k].double().cpu().numpy().reshape(spec.n, order="F")
        b = s64[k].cpu().numpy().reshape(spec.n, order="F")
        worst_rel = max(worst_rel, float(np.max(np.abs(a - b)) / np.max(np.abs(b))))
        worst_cells = max(worst_cells, zero_set_displacement_cells(a, b))
    return {"workload": "air3D 101^3, 11 slices to tau = 2.8 (%d RK3 steps), FP32 against the FP64 solve"
                        % st["steps"],
            "max_abs_err_rel": worst_rel, "zero_set_displacement_cells": worst_cells,
            "bar_cells": 0.1}


def cpu_oracle_rate(spec, V0, steps: int):
    """The FP64 oracle, single-threaded, on the full 101^3 grid for `steps` RK3 steps."""
    from oracle import oracle as O
    m = O.method(scheme=O.WENO5, dynamics=O.DYN_AIR3D, params=(5.0, 5.0, 1.0, 1.0), brt=O.BRT_MIN0)
    dt = 0.8 / O.step_bound_inv(spec, m)
    V = V0
    t0 = time.perf_counter()
    for _ in range(steps):
        V = O.rk3_step(spec, m, V, dt)
    el = time.perf_counter() - t0
    return steps * N_CELLS / el, el


def host_cores() -> int:
    """Host cores this process may run on (at most 64: each oracle process holds
    about 100 MB)."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    return max(1, min(n, 64))


_start_barrier = None


def _oracle_worker_init(barrier):
    global _start_barrier
    _start_barrier = barrier


def _oracle_worker(job):
    """One process of the all-core oracle run: W untimed then K timed RK3 steps
    of the full grid, started together with the other workers."""
    warmup, steps = job
    from oracle import oracle as O
    spec, V0 = workload()
    m = O.method(scheme=O.WENO5, dynamics=O.DYN_AIR3D, params=(5.0, 5.0, 1.0, 1.0), brt=O.BRT_MIN0)
    dt = 0.8 / O.step_bound_inv(spec, m)
    V = V0
    for _ in range(warmup):
        V = O.rk3_step(spec, m, V, dt)
    _start_barrier.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        V = O.rk3_step(spec, m, V, dt)
    return time.perf_counter() - t0


def cpu_oracle_rate_all_cores(warmup: int, steps: int, procs: int):
    """The unmodified oracle on every host core: `procs` spawned processes, each
    stepping its own copy of the grid (the oracle is single-threaded, so the
    grids are the unit of parallel work). Returns (aggregate cell-updates/s,
    slowest worker's timed seconds)."""
    import multiprocessing as mp
    from oracle import oracle as O
    O.build()
    mpc = mp.get_context("spawn")
    barrier = mpc.Barrier(procs)
    with mpc.Pool(procs, initializer=_oracle_worker_init, initargs=(barrier,)) as pool:
        els = pool.map(_oracle_worker, [(warmup, steps)] * procs, chunksize=1)
    el = max(els)
    return procs * steps * N_CELLS / el, el


def run_reference(args, world, rank):
    if rank != 0:
        return
    procs = host_cores()
    value, el = cpu_oracle_rate_all_cores(args.warmup, args.steps, procs)
    line = {"impl": "reference", "metric": "cell-updates/s (air3D 101^3 WENO5 TVD-RK3 step)", "value": value,
            "unit": "cell-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "air3d-101^3 WENO5 LF TVD-RK3 CFL0.8 BRT-min0", "cells": N_CELLS,
                       "l2": "host run (no GPU)"},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": procs, "kind": "oracle",
                             "sample": "%d RK3 steps of the full 101^3 grid in each of %d processes (one per "
                                       "host core, the unmodified single-threaded oracle each)" % (args.steps, procs)},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=24, help="oracle steps for the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--legs", default="f64,f32,e2e,batch,serve,large",
                    help="comma list of legs to run; f64 always runs, and a run without all of them "
                         "(a profiling run: --legs f64, f64,f32, f64,large or f64,batch) prints timings instead of "
                         "the JSON line")
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--large-cases", default=None,
                    help="comma list of the large-grid cases to run in a partial run (default: all), e.g. "
                         "sphere512_f32,sphere512_f32_eno1,sphere512_f32_eno2,dubins81_f32,dubins81_f64")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    from paper_2507_11542_gb300 import _lib, build, solver
    if world == 1 and build.stale():
        build.build()
    torch.cuda.set_device(local)
    spec, V0 = workload()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    ctx = solver.Context(local)
    K, W_ = args.steps, max(args.warmup, 3)
    legs = set(args.legs.split(","))
    full = {"f32", "e2e", "batch", "serve", "large"} <= legs
    with ClockSampler(local) as clk:
        r64 = bench_dtype(ctx, spec, V0, "float64", K, W_, world, flush)
        r32 = bench_dtype(ctx, spec, V0, "float32", K, W_, world, flush) if "f32" in legs else None
        if not full:
            # a partial run (profiling): the chosen device legs only, no JSON line
            print("f64 leg: %.3f ms per step" % r64["ms_per_step"], flush=True)
            if r32:
                print("f32 leg: %.3f ms per step" % r32["ms_per_step"], flush=True)
            if "large" in legs:
                only = set(args.large_cases.split(",")) if args.large_cases else None
                print("large grids: %s" % json.dumps(bench_large(ctx, world, flush, only)), flush=True)
            if "batch" in legs:
                print("batched: %s" % json.dumps(bench_batch(ctx, rank=rank, world=world)), flush=True)
            if "serve" in legs:
                print("served: %s" % json.dumps(bench_serve(ctx, args.serve_requests)), flush=True)
            ctx.close()
            return
        e2e = bench_e2e(ctx, spec, V0, "float64", max(3, K // 4), 2, world)
        batch = bench_batch(ctx, rank=rank, world=world)
        serve = bench_serve(ctx, args.serve_requests) if world == 1 else None
        large = bench_large(ctx, world, flush)
        rockets = bench_rockets(ctx) if world == 1 else None
        fp32_error = bench_fp32_error(ctx, spec, V0) if world == 1 else None
    peaks = alu_peaks(local)
    hbm, hbm_kind = measured_hbm_gbs()
    value = world * K * N_CELLS / (r64["total_ms"] / 1e3)

    def roofline(r, dtype):
        launch_s = r["launch_ms_mean"] / 1e3
        tflops = FLOPS_PER_NODE_STAGE * N_CELLS / launch_s / 1e12
        es = 8 if dtype == "float64" else 4
        gbs = WORDS_PER_NODE_STEP / 3.0 * es * N_CELLS / launch_s / 1e9
        pk = peaks[dtype]
        return {"bound": "alu", "achieved": tflops, "peak": pk["measured_tflops"], "unit": "TFLOP/s",
                "frac": tflops / pk["measured_tflops"], "traffic": NCU_TRAFFIC_BYTES[dtype],
                "peak_source": "measured in this run: %s throughput probe (libhj_peak.so), best of 5 launches"
                               % ("DFMA" if dtype == "float64" else "FFMA"),
                "peak_unit_counts": pk["unit_count_tflops"], "peak_unit_counts_source": pk["unit_count_source"],
                "frac_of_unit_counts": tflops / pk["unit_count_tflops"],
                "flops_per_node": FLOPS_PER_NODE_STAGE,
                "flops_note": "two-sided WENO5 per dimension as the method states it (the kernel evaluates each "
                              "interface once for its two nodes); achieved = flops x 1,030,301 nodes / mean "
                              "stage-launch time (CUDA events on the launching stream)",
                "kernel": "rows_kernel<%s,3,AIR3D,WENO5> (fused stage)" % ("double" if dtype == "float64" else "float"),
                "launch_ms_mean": r["launch_ms_mean"],
                "hbm_achieved_gbs": gbs, "hbm_peak_gbs": hbm, "hbm_peak_source": hbm_kind, "hbm_frac": gbs / hbm}

    line = {
        "metric": "cell-updates/s (air3D 101^3 WENO5 TVD-RK3 step)",
        "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": K, "warmup": W_,
        "ms_per_step": r64["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "air3d-101^3 WENO5 LF TVD-RK3 CFL0.8 BRT-min0 FP64", "cells": N_CELLS,
                   "l2": "flushed (256 MiB write) before every timed step",
                   "time": "FP64 t, dt and CFL bound", "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roofline(r64, "float64"),
        "fp32": {"value": world * K * N_CELLS / (r32["total_ms"] / 1e3), "unit": "cell-updates/s",
                 "ms_per_step": r32["ms_per_step"], "steps": K, "roofline": roofline(r32, "float32"),
                 "error": fp32_error},
        "e2e": {k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")},
        "gpu_launches": r64["launches"],
        "clocks": clk.summary(),
        "alu_peaks": peaks,
    }
    line["e2e"]["rk3_steps_per_call"] = e2e["rk3_steps_per_step"]
    line["e2e"]["dtype"] = "f64"
    if batch:
        line["batched"] = batch
    if serve:
        line["served"] = serve
    line["large_grids"] = large
    if rockets:
        line["rockets"] = rockets
    if rank == 0 and world == 1 and not args.no_cpu_baseline:  # the host baseline is taken at N = 1 only
        rate1, el1 = cpu_oracle_rate(spec, V0, args.cpu_steps)
        procs = host_cores()
        rate, el = cpu_oracle_rate_all_cores(1, max(2, args.cpu_steps // 4), procs)
        line["cpu_baseline"] = {"value": rate, "unit": "cell-updates/s", "cores": procs, "kind": "oracle",
                                "sample": "%d RK3 steps of the full 101^3 air3D grid, FP64, in each of %d spawned "
                                          "processes (one per host core; the unmodified single-threaded oracle "
                                          "each, %.1f s)" % (max(2, args.cpu_steps // 4), procs, el),
                                "single_thread": {"value": rate1, "cores": 1,
                                                  "sample": "%d RK3 steps, one thread (%.1f s)" % (args.cpu_steps, el1)}}
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
