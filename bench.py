#!/usr/bin/env python
"""Throughput of the TDGL + Poisson step in cell-steps/s on GB300.

One "step" is one forward-Euler time step of a whole film: the warm-started
Poisson solve (to the workload's tolerance) followed by the TDGL update, all
in the CUDA library behind include/pf.h.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank advances its own film
(independent replicas, no collective on the data path); value = all ranks'
cell-steps / max over ranks of the timed device time ("scaling": "weak").
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TDGL cell-steps/s incl. Poisson solve"
UNIT = "cell-steps/s"
L2_BYTES = 129 * 2 ** 20
WORKLOADS = ("tip", "strips", "grounded", "batch", "adjoint", "air")


def make_workload(name, seed_offset=0, solver=None, size=None):
    from paper_1202_6116_gb300 import workloads as W
    dims = {} if size is None else dict(zip(("nx", "ny", "nz"), size))
    if name == "strips":
        w = W.film_strip_fp32(seed=1 + seed_offset, **dims)
    elif name == "tip":
        w = W.film_tip_fp32(seed=2 + seed_offset, **dims)
    elif name == "grounded":
        w = W.film_fp64_grounded(seed=0 + seed_offset, **dims)
    elif name == "air":
        w = W.film_open_air(seed=5 + seed_offset, **dims)
    else:
        raise ValueError(name)
    if solver == "mg":
        w = w.with_(solver="mg", maxit=500)      # MG-PCG needs tens of iterations, not thousands
    elif solver:
        w = w.with_(solver=solver)
    return w


def sample_workload(name):
    """Bounded CPU sample of a workload: the same recipe on a smaller film."""
    from paper_1202_6116_gb300 import workloads as W
    if name == "strips":
        return W.film_strip_fp32(64, 64, 16, seed=1), "64x64x16 film of the strip-electrode recipe"
    if name == "tip":
        return W.film_tip_fp32(128, 128, 16, seed=2), "128x128x16 film of the tip-electrode recipe"
    if name == "air":
        return W.film_open_air(32, 32, 21, seed=5), "32x32x21 film of the open-air recipe"
    return W.film_fp64_grounded(32, 32, 32, seed=0), "the full 32x32x32 grounded film"


def workload_config(w, name, flush, args=None):
    c = {"workload": "%s %dx%dx%d %s %s rtol=%g dt=%g" % (name, w.nx, w.ny, w.nz, w.precision,
                                                          "MG-PCG" if w.solver == "mg" else "Jacobi-PCG",
                                                          w.rtol, w.dt),
         "cells": w.n, "precision": w.precision, "solver": w.solver, "poisson_rtol": w.rtol,
         "dt": w.dt, "l2": flush}
    if args is not None:
        c["integrator"] = args.integrator
        c["poisson_every"] = max(1, args.poisson_every)
        order = args.extrap_order or (1 if args.noise > 0 else 2 if w.rtol > 5e-7 else 3)
        c["warm_start"] = ("last potential" if args.warm_last else
                           "extrapolated (order %d from the last potentials, compensated in FP32)" % order)
        if args.noise > 0:
            c["noise_sigma"] = args.noise
        if w.n_air:
            c["n_air"] = w.n_air
    return c


# --------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ roofline

def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Device-code sources of each kernel family (the files that define it; the
# shared march, reduction and layout headers belong to every family).
FAMILY_SOURCES = {
    "cg": ("pf_cg.cu",),
    "mg": ("pf_mg.cu",),
    "step": ("pf_step.cu", "pf_rng.cuh"),
    "flat": ("pf_kernels.cu",),
    "diag": ("pf_diag.cu",),
    "adj": ("pf_adjoint.cu",),
}
COMMON_SOURCES = ("pf_march.cuh", "pf_common.cuh", "pf_internal.h")


def family_of(kernel):
    name = kernel.split(".")[0]
    if name.startswith("mg_"):
        return "mg"
    if name in ("cg_p", "cg_r"):
        return "cg"
    if name in ("cg_finish", "extrap", "sub_mean", "invdiag"):
        return "flat"
    if name == "diag":
        return "diag"
    if name == "tdgl_adj":
        return "adj"
    return "step"


def _code_only(text):
    """Source text without comments and blank space (edits of comments leave
    the compiled kernel, and so the hash, unchanged)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash(kernel):
    """Hash of the device code that defines a kernel family."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1202_6116_gb300", "csrc")
    for f in sorted(FAMILY_SOURCES[family_of(kernel)] + COMMON_SOURCES):
        h.update(_code_only(open(os.path.join(csrc, f)).read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload, cells):
    """DRAM bytes per launch of a kernel family from the committed ncu summary,
    scaled to this workload's cell count; None if absent or taken on other code."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    e = d.get("kernels", {}).get(kernel)
    if not e or e.get("workload") != workload or e.get("source_hash") != kernel_source_hash(kernel):
        return None
    return e["dram_bytes_per_cell"] * cells


# ------------------------------------------------------------ replicas (N > 1)

def replica_throughput(ms_local, cell_steps_local, world, device=None):
    """Whole-job throughput of N independent replicas (one film per rank, no
    collective on the data path): every rank did the same work, so value =
    N x local cell-steps / the slowest rank's time.  Returns (max ms, value);
    with world > 1 the MAX is an all-reduce over the default process group."""
    ms_max = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_max], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    return ms_max, cell_steps_local * world / (ms_max / 1e3)


# ------------------------------------------------------------------ our impl

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1202_6116_gb300 import build as B
    from paper_1202_6116_gb300 import pf
    from paper_1202_6116_gb300.film import Film

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = make_workload(args.workload, seed_offset=rank, solver=args.solver, size=args.size)
    if args.dt:
        w = w.with_(dt=args.dt)
    over = {"flags": (pf.PF_FLAG_NO_GRAPHS if args.no_graphs else 0) | (pf.PF_FLAG_WARM_LAST if args.warm_last else 0),
            "integrator": pf.PF_HEUN if args.integrator == "heun" else pf.PF_EULER,
            "poisson_every": args.poisson_every, "extrap_order": args.extrap_order}
    film = Film(w, device=dev, **over)
    if args.noise > 0:
        film.set_noise(args.noise, 12345)
    stream = film.stream
    flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    flush = "flushed (a %d MiB buffer is written between timed steps)" % (2 * L2_BYTES // 2 ** 20)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        film.step(1)
    clocks = ClockSampler(local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches = 0
    iters = 0
    graph_steps = 0
    barrier()
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush_buf.zero_()
        starts[k].record(stream)
        st, info = film.step(1)
        ends[k].record(stream)
        launches += info["kernel_launches"]
        iters += info["total_iters"]
        graph_steps += info["graph_steps"]
    barrier()
    clk = clocks.stop()
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    ms_max, value = replica_throughput(ms, w.n * args.steps, world, dev)

    # per-kernel device times: a second pass of the same steps with the
    # library's CUDA-event profiler on (kept out of the headline timing)
    prof_steps = max(1, min(args.steps, args.profile_steps))
    pf.pf_profile_enable(film.ctx, 1)
    barrier()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    prof_ms = 0.0
    for k in range(prof_steps):
        flush_buf.zero_()
        p0.record(stream)
        film.step(1)
        p1.record(stream)
        p1.synchronize()
        prof_ms += p0.elapsed_time(p1)
    stats = pf.pf_profile_read(film.ctx)
    pf.pf_profile_enable(film.ctx, 0)

    # end to end: host-resident state, copies inside the timed region
    w_bytes = 4 if w.precision == "fp32" else 8
    tdt = torch.float32 if w.precision == "fp32" else torch.float64
    Ph = film.P.detach().to("cpu").pin_memory()
    phih = film.phi.detach().to("cpu").pin_memory()
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    film.step(1)
    barrier()
    t0 = time.perf_counter()
    pf.pf_step_host(film.ctx, Ph, phih, e2e_steps)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    e2e_ms, e2e_value = replica_throughput(1e3 * e2e_s, w.n * e2e_steps, world, dev)
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": 4 * w.n * w_bytes, "d2h_bytes_per_step": 4 * w.n * w_bytes,
           "steps": e2e_steps}

    # roofline of the dominant kernel family (live CUDA-event times)
    work = [s for s in stats if s["launches"] > 0]
    dom = max(work, key=lambda s: s["total_ms"])
    total_kernel_ms = sum(s["total_ms"] for s in work)
    peak, peak_kind = measured_peak_hbm()
    achieved = dom["bytes"] / (dom["total_ms"] / 1e3) / 1e9
    traffic = ncu_traffic(dom["name"], args.workload, w.n)
    roofline = {"bound": "hbm", "kernel": dom["name"], "achieved": round(achieved, 1), "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": traffic,
                "algorithmic_bytes_per_launch": dom["bytes"] / dom["launches"],
                "avg_launch_us": 1e3 * dom["total_ms"] / dom["launches"],
                "share_of_kernel_time": round(dom["total_ms"] / total_kernel_ms, 3),
                "step_achieved_gbs": round(sum(s["bytes"] for s in work) / (total_kernel_ms / 1e3) / 1e9, 1),
                "profiled_steps": prof_steps, "profiled_ms_per_step": prof_ms / prof_steps,
                "kernels": {s["name"]: {"launches": s["launches"], "idle": s["idle_launches"],
                                        "ms": round(s["total_ms"], 3),
                                        "gbs": round(s["bytes"] / (s["total_ms"] / 1e3) / 1e9, 1)}
                            for s in work}}

    cpu = None
    film.close()
    prec = None
    if rank == 0 and world == 1 and args.precision_steps > 3:
        prec = precision_check(dev, args.precision_steps)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, args.cpu_seconds)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if w.precision == "fp32" else "f64",
                "data": "synthetic (seeded SplitMix64 initial state, electrode masks of the workload)",
                "config": workload_config(w, args.workload, flush, args),
                "poisson_iters_per_step": iters / args.steps,
                "graph_steps": graph_steps,
                "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
                "clocks": clk, "fp32_vs_fp64": prec, "impl": "ours"}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------- batched film sweep

def run_batch(args):
    """64 independent FP32 films (32^3 .. 128x128x64, CG to 1e-6 with the
    multigrid preconditioner, or Jacobi with --solver pcg; triangular
    top-electrode ramps) advanced together: one CUDA graph launch per batch
    step.  Tilings from the autotuner, per film shape."""
    import numpy as np
    import torch

    from paper_1202_6116_gb300 import autotune as AT
    from paper_1202_6116_gb300 import build as B
    from paper_1202_6116_gb300 import pf
    from paper_1202_6116_gb300 import workloads as W
    from paper_1202_6116_gb300.batch import Batch
    from paper_1202_6116_gb300.film import Film

    B.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ws = W.film_batch_hysteresis(nfilms=args.films, seed=4, steps=args.steps + args.warmup)
    if args.solver != "pcg":                       # multigrid-preconditioned CG unless Jacobi is asked for
        ws = [w.with_(solver="mg", maxit=500) for w in ws]
    t0 = time.perf_counter()
    tuned = {}
    for w in ws:
        k = AT.key_of(w)
        if k not in tuned:
            tuned[k] = AT.tune(w, steps=3, warmup=1, device=dev)
    tune_s = time.perf_counter() - t0
    films = [Film(w, device=dev, extrap_order=args.extrap_order) for w in ws]
    for f in films:
        AT.apply(f, tuned[AT.key_of(f.w)])
    record_every = 10
    b = Batch(films, max_records=(args.steps + args.warmup) // record_every + 1, record_every=record_every)
    for i, w in enumerate(ws):
        b.set_ramp(i, pf.PF_ZHI, *w.extra["ramp"])
    stream = films[0].stream
    b.step(args.warmup)
    clocks = ClockSampler(0)
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st, info = b.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    cells = sum(w.n for w in ws)
    loops = b.loops()
    b.close()
    # the same films stepped one after another (one graph launch per film and step)
    seq_steps = max(1, min(10, args.steps))
    torch.cuda.synchronize(dev)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    seq_iters = 0
    for _ in range(seq_steps):
        for f in films:
            _, fi = f.step(1, ok=(pf.PF_OK, pf.PF_ERR_NOCONV))
            seq_iters += fi["total_iters"]
    s1.record(stream)
    s1.synchronize()
    seq_ms = s0.elapsed_time(s1)
    for f in films:
        f.close()
    value = cells * args.steps / (ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded SplitMix64 initial states and ramp draws)",
            "config": {"workload": "batch of %d FP32 films (32^3, 64x64x32, 96x96x48, 128x128x64 drawn with "
                                   "seed 4), grounded bottom, ramped top electrode, %s rtol=1e-06 dt=0.01"
                                   % (len(ws), "MG-PCG" if ws[0].solver == "mg" else "Jacobi-PCG"),
                       "cells": cells, "films": len(ws), "solver": ws[0].solver,
                       "extrap_order": args.extrap_order or (2 if ws[0].rtol > 5e-7 else 3),
                       "l2": "inputs larger than L2 (%.2f GB of film state)" % (cells * 4 * 11 / 1e9)},
            "poisson_iters_per_step": info["total_iters"] / args.steps / len(ws),
            "gpu_launches": info["kernel_launches"], "status": pf.STATUS_NAMES[st],
            "sequential_ms_per_step": seq_ms / seq_steps,
            "sequential_iters_per_film_step": seq_iters / seq_steps / len(ws),
            "batch_speedup_vs_sequential": round((seq_ms / seq_steps) / (ms / args.steps), 3),
            "autotune": {k: {"vx": v["vx"], "tz": v["tz"], "blocks_per_sm": v["blocks_per_sm"],
                             "us_per_iter": round(1e3 * v["ms_per_iter"], 2),
                             "default_us_per_iter": round(1e3 * v["default_ms_per_iter"], 2)}
                         for k, v in tuned.items()},
            "autotune_seconds": round(tune_s, 1),
            "loop_records": int(loops.shape[0]),
            "loop_example": {"film": 0, "volts": [round(x, 4) for x in loops[:, 0, 0][-5:].tolist()],
                             "mean_pz": [round(x, 5) for x in loops[:, 0, 3][-5:].tolist()]},
            "clocks": clk, "impl": "ours"}
    print(json.dumps(line))


# ------------------------------------------------- differentiation workload

def run_adjoint(args):
    """Gradient of the differentiation workload (128x128x32 FP64, strip
    electrodes, 500 steps, MG-PCG to 1e-12) through the discrete adjoint: forward pass with a
    checkpoint every 50 steps, backward pass recomputing each segment.  The
    metric counts forward cell-steps of the trajectory per second of the whole
    forward + backward computation."""
    import torch

    from paper_1202_6116_gb300 import adjoint as A
    from paper_1202_6116_gb300 import build as B
    from paper_1202_6116_gb300 import workloads as W

    B.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = W.film_adjoint_fp64().with_(solver="mg", maxit=500)
    steps = args.steps
    spec = A.TrajectorySpec(w, steps=steps, checkpoint_every=50, device="cuda")
    P0 = torch.as_tensor(w.P0, device=dev)
    target = torch.zeros_like(P0)
    target[2] = 1.0

    def one():
        coeffs = torch.tensor([w.a1, w.a11, w.a12, w.g], dtype=torch.float64, device=dev, requires_grad=True)
        vlo = torch.as_tensor(w.volt_lo, device=dev).clone().requires_grad_(True)
        vhi = torch.as_tensor(w.volt_hi, device=dev).clone().requires_grad_(True)
        P = A.trajectory(P0, coeffs, vlo, vhi, spec)
        loss = ((P[2] - target[2]) ** 2).mean()
        loss.backward()
        return coeffs.grad.detach().cpu().numpy()

    for _ in range(max(1, args.warmup // 3)):
        one()
    clocks = ClockSampler(0)
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.3)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    grad = one()
    e1.record(stream)
    e1.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    line = {"metric": "TDGL cell-steps/s of forward + discrete adjoint (gradient of a trajectory)",
            "value": w.n * steps / (wall), "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wall / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (seeded SplitMix64 initial state, strip electrodes)",
            "config": {"workload": "adjoint 128x128x32 fp64 MG-PCG rtol=1e-12 dt=0.01, checkpoint every 50",
                       "cells": w.n, "loss": "mean (P_z - 1)^2 of the final state"},
            "device_ms": ms, "grad_a1_a11_a12_g": [float(v) for v in grad], "clocks": clk, "impl": "ours"}
    print(json.dumps(line))


# -------------------------------------------------------- FP32 against FP64

def precision_check(dev, steps):
    """The strip-electrode film (256x256x64, MG-PCG to 1e-8) advanced in FP32
    (FP64 reductions) and in plain FP64 on this GPU: time per step of each,
    the FP32 error on P (max |P32 - P64| / max |P64| per component) and the
    switched-domain fraction (P_x > 0.3) of both."""
    import torch
    from paper_1202_6116_gb300 import workloads as W
    from paper_1202_6116_gb300.film import Film
    out = {"workload": "strips 256x256x64 MG-PCG rtol=1e-08 dt=0.01, %d steps from the seeded state" % steps}
    finals = {}
    for prec in ("fp32", "fp64"):
        w = W.film_strip_fp32().with_(precision=prec, solver="mg", maxit=500)
        f = Film(w, device=dev)
        f.step(3)                                  # graph capture and warm-up, excluded
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(f.stream)
        _, info = f.step(steps - 3)
        e1.record(f.stream)
        e1.synchronize()
        d = f.diagnostics(0.3)
        finals[prec] = f.P.double()
        out[prec + "_ms_per_step"] = round(e0.elapsed_time(e1) / (steps - 3), 4)
        out[prec + "_poisson_iters_per_step"] = round(info["total_iters"] / (steps - 3), 2)
        out[prec + "_switched_fraction"] = d["switched_fraction"]
        f.close()
    a, b = finals["fp32"], finals["fp64"]
    out["max_rel_err_P"] = max(float((a[c] - b[c]).abs().max() / b[c].abs().max()) for c in range(3))
    out["switched_diff_pp"] = 100.0 * abs(out["fp32_switched_fraction"] - out["fp64_switched_fraction"])
    out["fp32_speedup"] = round(out["fp64_ms_per_step"] / out["fp32_ms_per_step"], 3)
    return out


# ----------------------------------------------------------------- CPU oracle

def oracle_timed(w, warm, steps):
    import oracle as O
    G = O.Grid(w.nx, w.ny, w.nz, w.dx, w.periodic_z, w.type_lo, w.volt_lo, w.type_hi, w.volt_hi, w.eps)
    prm = O.Params(w.a1, w.a11, w.a12, w.g, w.L, w.dt, w.rtol, w.maxit)
    P, phi, _, _ = O.step(G, prm, w.P0, None, warm)
    t0 = time.perf_counter()
    P, phi, st, info = O.step(G, prm, P, phi, steps)
    return time.perf_counter() - t0, info


def cpu_baseline(name, budget_s):
    """The FP64 oracle as it stands, serial, on a bounded sample of the workload."""
    import oracle.build
    oracle.build.build()
    w, desc = sample_workload(name)
    dt1, _ = oracle_timed(w, 2, 1)
    steps = max(1, min(50, int(budget_s / max(dt1, 1e-3))))
    secs, info = oracle_timed(w, 2, steps)
    return {"value": w.n * steps / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%s, FP64, %d timed steps after 3 warm-up steps (%.1f s, %d CG iterations)" %
                      (desc, steps, secs, info["total_iters"])}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import oracle.build
    oracle.build.build()
    w, desc = sample_workload(args.workload)
    secs, info = oracle_timed(w, args.warmup, args.steps)
    value = w.n * args.steps / secs
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64 initial state, electrode masks of the workload)",
            "config": workload_config(make_workload(args.workload, solver=args.solver, size=args.size), args.workload,
                                      "n/a (CPU)"),
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%s, FP64 serial oracle, %d steps after %d warm-up steps" %
                                       (desc, args.steps, args.warmup)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--workload", choices=WORKLOADS, default="tip")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--solver", choices=("pcg", "mg"), default=None,
                    help="override the workload's Poisson preconditioner (Jacobi or multigrid)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--profile-steps", type=int, default=10)
    ap.add_argument("--size", type=lambda v: tuple(int(x) for x in v.lower().split("x")), default=None,
                    help="NXxNYxNZ: the workload's recipe on another grid (profiling runs)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--precision-steps", type=int, default=200,
                    help="steps of the FP32-against-FP64 comparison on the strip film (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--films", type=int, default=64, help="films of the batch workload")
    ap.add_argument("--integrator", choices=("euler", "heun"), default="euler",
                    help="forward Euler or the paper's predictor-corrector")
    ap.add_argument("--poisson-every", type=int, default=1, help="solve the potential on every k-th step only")
    ap.add_argument("--dt", type=float, default=None, help="override the workload's time step")
    ap.add_argument("--noise", type=float, default=0.0, help="thermal random force sigma (0: off)")
    ap.add_argument("--extrap-order", type=int, choices=(0, 1, 2, 3), default=0,
                    help="highest order of the extrapolated start (0: automatic)")
    ap.add_argument("--warm-last", action="store_true",
                    help="start each solve from the last potential (the paper's scheme) instead of extrapolating")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch every kernel from the host (profilers cannot see kernels inside CUDA graphs "
                         "with conditional nodes)")
    args = ap.parse_args()
    if args.impl == "reference":
        args.steps = 5 if args.steps is None else args.steps
        args.warmup = 3 if args.warmup is None else args.warmup
        run_reference(args)
    elif args.workload == "batch":
        args.steps = 300 if args.steps is None else args.steps
        args.warmup = 5 if args.warmup is None else max(3, args.warmup)
        run_batch(args)
    elif args.workload == "adjoint":
        args.steps = 500 if args.steps is None else args.steps
        args.warmup = 3 if args.warmup is None else max(3, args.warmup)
        run_adjoint(args)
    else:
        args.steps = 30 if args.steps is None else args.steps
        args.warmup = 5 if args.warmup is None else max(3, args.warmup)
        run_ours(args)


if __name__ == "__main__":
    main()
