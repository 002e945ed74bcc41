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
import contextlib
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
    state_gb = (4 * w.n * (4 if w.precision == "fp32" else 8) + film.ws_bytes) / 1e9
    flush = ("inputs larger than L2: every step streams the film's fields (%.2f GB of state and workspace, "
             "L2 %d MiB)" % (state_gb, L2_BYTES // 2 ** 20))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        film.step(1)
    clocks = ClockSampler(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    clocks.start()
    time.sleep(0.3)
    # the K steps go out as one asynchronous call: one CUDA graph per step,
    # no host round trip between steps, the statistics read once at the end
    e0.record(stream)
    film.step_async(args.steps)
    e1.record(stream)
    st, info = film.wait()
    barrier()
    clk = clocks.stop()
    launches = info["kernel_launches"]
    iters = info["total_iters"]
    graph_steps = info["graph_steps"]
    ms = e0.elapsed_time(e1)
    ms_max, value = replica_throughput(ms, w.n * args.steps, world, dev)

    # per-kernel device times: a second pass of the same steps with the
    # library's CUDA-event profiler on (kept out of the headline timing)
    prof_steps = max(1, min(args.steps, args.profile_steps))
    pf.pf_profile_enable(film.ctx, 1)
    barrier()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    prof_ms = 0.0
    # an NVTX range around exactly these steps, so that an ncu launch list
    # (--nvtx --nvtx-include "pf_profile_steps/") covers the same launches
    torch.cuda.nvtx.range_push("pf_profile_steps")
    for k in range(prof_steps):
        flush_buf.zero_()
        p0.record(stream)
        film.step(1)
        p1.record(stream)
        p1.synchronize()
        prof_ms += p0.elapsed_time(p1)
    torch.cuda.nvtx.range_pop()
    stats = pf.pf_profile_read(film.ctx)
    pf.pf_profile_enable(film.ctx, 0)

    # end to end: host-resident state, copies inside the timed region
    w_bytes = 4 if w.precision == "fp32" else 8
    tdt = torch.float32 if w.precision == "fp32" else torch.float64
    Ph = film.P.detach().to("cpu").pin_memory()
    phih = film.phi.detach().to("cpu").pin_memory()
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    # untimed warm-up through the same call: its steps alternate the two
    # polarization buffers, whose one-step graphs are captured on first use
    e2e_warm = 2
    pf.pf_step_host(film.ctx, Ph, phih, e2e_warm)
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    pf.pf_step_host(film.ctx, Ph, phih, e2e_steps)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    e2e_ms, e2e_value = replica_throughput(1e3 * e2e_s, w.n * e2e_steps, world, dev)
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": 4 * w.n * w_bytes, "d2h_bytes_per_step": 4 * w.n * w_bytes,
           "steps": e2e_steps, "warmup": e2e_warm}

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
    full = None
    if rank == 0 and world == 1 and args.precision_steps > 3:
        prec = precision_check(dev, args.precision_steps)
    if rank == 0 and world == 1 and args.full_steps > 4 and args.workload == "tip":
        full = full_run(dev, w, args.full_steps)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, args.cpu_seconds)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if w.precision == "fp32" else "f64",
                "data": "synthetic (seeded SplitMix64 initial state, electrode masks of the workload)",
                "config": workload_config(w, args.workload, flush, args),
                "poisson_iters_per_step": iters / args.steps,
                "max_poisson_iters": info["max_iters"],
                "graph_steps": graph_steps,
                "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
                "clocks": clk, "fp32_vs_fp64": prec, "full_run": full, "impl": "ours"}
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

def precision_check(dev, steps, chunk=1000):
    """The strip-electrode film (256x256x64, MG-PCG to 1e-8) advanced for
    the whole run in FP32 (the compensated state, the default), in plain
    FP32 and in FP64 on this GPU, side by side in chunks: time per step of
    each, the FP32 errors on P against FP64 after every chunk (max |P32 -
    P64| / max |P64| per component, the maximum over components; the
    relative 2-norm error; the cells off by more than 1e-4), the
    switched-domain fraction (P_x > 0.3) of each, and the true FP64 residual
    of each run's last potential."""
    import torch
    from paper_1202_6116_gb300 import pf
    from paper_1202_6116_gb300 import workloads as W
    from paper_1202_6116_gb300.film import Film
    out = {"workload": "strips 256x256x64 MG-PCG rtol=1e-08 dt=0.01, %d steps from the seeded state" % steps,
           "error_metric": "max |P32 - P64| / max |P64| per component (the maximum over components)",
           "references": "fp64: from the seeded state; fp64_rounded_start: from the seeded state rounded to "
                         "FP32, the values the FP32 runs start from"}
    # fp64_rounded_start: FP64 from the initial state rounded to FP32 -- how
    # far the dynamics carry a perturbation of one FP32 rounding by itself
    forms = (("fp32", "fp32", 0), ("fp32_plain", "fp32", pf.PF_FLAG_PLAIN_FP32), ("fp64", "fp64", 0),
             ("fp64_rounded_start", "fp64", 0))
    films, ms, its, solves, worst = {}, {}, {}, {}, {}
    for key, prec, flags in forms:
        w = W.film_strip_fp32().with_(precision=prec, solver="mg", maxit=500)
        if key == "fp64_rounded_start":
            w = w.with_(P0=w.P0.astype("float32").astype("float64"))
        films[key] = Film(w, device=dev, flags=flags)
        films[key].step(3)                         # graph captures and warm-up, excluded from the timing
        ms[key], its[key], solves[key], worst[key] = 0.0, 0, 0, 0
    done = 3
    timeline = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    while done < steps - 1:
        n = min(chunk - done % chunk, steps - 1 - done)
        for key, f in films.items():
            torch.cuda.synchronize(dev)
            e0.record(f.stream)
            f.step_async(n)
            e1.record(f.stream)
            _, info = f.wait()
            ms[key] += e0.elapsed_time(e1)
            its[key] += info["total_iters"]
            solves[key] += info["solves"]
            worst[key] = max(worst[key], info["max_iters"])
        done += n
        if done % chunk == 0 or done == steps - 1:
            b = films["fp64"].P
            b0 = films["fp64_rounded_start"].P
            row = {"step": done}
            for key in ("fp32", "fp32_plain", "fp64_rounded_start"):
                a = films[key].P.double()
                row[key] = max(float((a[c] - b[c]).abs().max() / b[c].abs().max()) for c in range(3))
            for key in ("fp32", "fp32_plain"):
                a = films[key].P.double()
                row[key + "_vs_rounded_start"] = max(float((a[c] - b0[c]).abs().max() / b0[c].abs().max())
                                                     for c in range(3))
            timeline.append(row)
    finals = {}
    for key, f in films.items():
        Pprev = f.P.clone()
        f.step(1)                                  # the last step: its potential belongs to Pprev
        res, bn, resc = f.true_residual(Pprev)
        d = f.diagnostics(0.3)
        finals[key] = f.P.double()
        out[key + "_ms_per_step"] = round(ms[key] / (steps - 4), 4)
        out[key + "_poisson_iters_per_step"] = round(its[key] / max(1, solves[key]), 3)
        out[key + "_max_poisson_iters"] = worst[key]
        out[key + "_switched_fraction"] = d["switched_fraction"]
        out[key + "_true_relres_last_solve"] = res / bn if bn > 0 else 0.0
        out[key + "_true_relres_last_solve_compensated"] = resc / bn if bn > 0 else 0.0
        f.close()
        del Pprev
    b = finals["fp64"]
    b0 = finals["fp64_rounded_start"]
    for key in ("fp32", "fp32_plain"):
        a = finals[key]
        out[key + "_max_rel_err_P_vs_rounded_start"] = max(float((a[c] - b0[c]).abs().max() / b0[c].abs().max())
                                                           for c in range(3))
    for key in ("fp32", "fp32_plain", "fp64_rounded_start"):
        a = finals[key]
        out[key + "_max_rel_err_P"] = max(float((a[c] - b[c]).abs().max() / b[c].abs().max()) for c in range(3))
        out[key + "_rel_l2_err_P"] = float((a - b).norm() / b.norm())
        out[key + "_cells_off_by_1e-4"] = int(((a - b).abs() > 1e-4).sum())
        out[key + "_switched_diff_pp"] = 100.0 * abs(out[key + "_switched_fraction"] - out["fp64_switched_fraction"])
        out[key + "_peak_max_rel_err_P"] = max([r[key] for r in timeline] + [out[key + "_max_rel_err_P"]])
    out["timeline"] = timeline
    out["max_rel_err_P"] = out["fp32_max_rel_err_P"]
    out["switched_diff_pp"] = out["fp32_switched_diff_pp"]
    out["fp32_speedup"] = round(out["fp64_ms_per_step"] / out["fp32_ms_per_step"], 3)
    out["fp32_peak_max_rel_err_P_vs_rounded_start"] = max(
        [r["fp32_vs_rounded_start"] for r in timeline] + [out["fp32_max_rel_err_P_vs_rounded_start"]])
    out["meets_stated_error"] = bool(out["fp32_peak_max_rel_err_P"] <= 1e-4 and out["switched_diff_pp"] <= 0.1)
    return out


def full_run(dev, w, steps):
    """One whole run of the bench film from its seeded state (untimed in the
    headline): Poisson iterations per step over all of it, device time per
    step, and the true FP64 relative residual ||b - A phi|| / ||b|| of the
    last solve (phi as stored, P the state it was solved for)."""
    import torch
    from paper_1202_6116_gb300.film import Film
    f = Film(w, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f.step(2)                                      # graph captures
    pairs = (steps - 4) // 2
    total, solves, worst, nonconv = 0, 0, 0, 0
    torch.cuda.synchronize(dev)
    ms = 0.0
    for _ in range(pairs):                         # two steps per call: the state ends in the bound buffer
        e0.record(f.stream)
        f.step_async(2)
        e1.record(f.stream)
        _, info = f.wait()
        ms += e0.elapsed_time(e1)
        total += info["total_iters"]
        solves += info["solves"]
        worst = max(worst, info["max_iters"])
        nonconv += info["nonconverged"]
    done = 2 + 2 * pairs
    while done < steps - 1:
        _, info = f.step(1)
        total, solves, worst, done = total + info["total_iters"], solves + info["solves"], \
            max(worst, info["max_iters"]), done + 1
    Pprev = f.P.clone()
    _, info = f.step(1)
    total, solves, worst = total + info["total_iters"], solves + info["solves"], max(worst, info["max_iters"])
    res, bn, resc = f.true_residual(Pprev)
    d = f.diagnostics(0.3)
    out = {"workload": "%s, %d steps from the seeded state" % (w.name, steps),
           "steps": steps, "poisson_iters_per_step_mean": round(total / max(1, solves), 3),
           "poisson_iters_per_step_max": worst, "nonconverged": nonconv,
           "ms_per_step_steps_3_to_%d" % (2 + 2 * pairs): round(ms / (2 * pairs), 4),
           "last_solve_recursive_relres": info["last_relres"],
           "last_solve_true_relres_fp64": {"stored_fp32_phi": res / bn if bn > 0 else 0.0,
                                           "compensated_phi": resc / bn if bn > 0 else 0.0},
           "mean_P": [d["mean_px"], d["mean_py"], d["mean_pz"]], "switched_fraction": d["switched_fraction"]}
    f.close()
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


def host_cpu():
    """Core count and CPU model of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"nproc": os.cpu_count(), "model": model or "unknown", "arch": platform.machine()}


def sample_desc(w, desc):
    return "%s (%dx%dx%d, FP64, Jacobi-PCG rtol=%g, dt=%g)" % (desc, w.nx, w.ny, w.nz, w.rtol, w.dt)


def oracle_rate(name, budget_s, openmp):
    """cell-steps/s of the FP64 oracle on the bounded sample: steps sized to
    about budget_s seconds of CPU work after 2 warm-up steps."""
    import oracle as O
    import oracle.build
    w, desc = sample_workload(name)
    ctx = O.openmp() if openmp else contextlib.nullcontext()
    with ctx:
        oracle.build.build(openmp=openmp)
        dt1, _ = oracle_timed(w, 2, 1)
        steps = max(1, min(200, int(budget_s / max(dt1, 1e-3))))
        secs, info = oracle_timed(w, 2, steps)
        cores = O.threads()
    return {"value": w.n * steps / secs, "unit": UNIT, "cores": cores,
            "kind": "oracle" + (" (OpenMP build)" if openmp else ""),
            "cflags": " ".join(oracle.build.flags(openmp)),
            "sample": "%s, %d timed steps after 2 warm-up steps (%.1f s, %d CG iterations)" %
                      (sample_desc(w, desc), steps, secs, info["total_iters"])}


def cpu_baseline(name, budget_s):
    """The FP64 oracle as it stands on a bounded sample of the workload: the
    serial build on one core, and the same source built with OpenMP on all
    of this host's cores."""
    base = oracle_rate(name, budget_s, openmp=False)
    base["host"] = host_cpu()
    base["all_cores"] = oracle_rate(name, budget_s, openmp=True)
    return base


def run_reference(args):
    """The reference arm: the FP64 oracle (the OpenMP build of the same
    source, on all host cores) on a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import oracle as O
    import oracle.build
    w, desc = sample_workload(args.workload)
    with O.openmp():
        oracle.build.build(openmp=True)
        secs, info = oracle_timed(w, args.warmup, args.steps)
        cores = O.threads()
    value = w.n * args.steps / secs
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64 initial state, electrode masks of the workload)",
            "config": {"workload": "%s %dx%dx%d fp64 Jacobi-PCG rtol=%g dt=%g (CPU oracle sample of the %s film)"
                                   % (args.workload, w.nx, w.ny, w.nz, w.rtol, w.dt, args.workload),
                       "cells": w.n, "precision": "fp64", "solver": "pcg", "poisson_rtol": w.rtol, "dt": w.dt,
                       "l2": "n/a (CPU)", "cores": cores},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle (OpenMP build)",
                             "cflags": " ".join(oracle.build.flags(True)), "host": host_cpu(),
                             "sample": "%s, %d steps after %d warm-up steps, %d CG iterations" %
                                       (sample_desc(w, desc), args.steps, args.warmup, info["total_iters"])},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# -------------------------------------------------- replica launch (N > 1)

def launch_replicas(args, argv):
    """Start N ranks of this script (one per GPU) with torch's launcher when
    --gpus N > 1 is asked for without one; rank 0 prints the line."""
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=%d" % args.gpus,
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + argv
    return subprocess.call(cmd)


def run_replica_selftest(args):
    """The multi-rank path of the bench without a GPU (gloo): every rank
    reports a fixed local time (10 ms x (rank + 1)) for a fixed amount of
    work, and rank 0 prints the whole-job line the GPU run would print."""
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        dist.init_process_group("gloo")
    cells, steps = 1000, args.steps
    ms_local = 10.0 * (rank + 1)
    ms_max, value = replica_throughput(ms_local, cells * steps, world)
    if rank == 0:
        print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
                          "ms_per_step": ms_max / steps, "scaling": "weak", "impl": "selftest"}))
    if world > 1:
        dist.destroy_process_group()


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
    ap.add_argument("--precision-steps", type=int, default=5000,
                    help="steps of the FP32-against-FP64 comparison on the strip film (0: skip)")
    ap.add_argument("--full-steps", type=int, default=1000,
                    help="steps of the untimed whole run of the tip film (iterations per step, true residual; 0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--replica-selftest", action="store_true",
                    help="exercise the multi-rank launch and reduction on CPU (gloo), no GPU work")
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
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(launch_replicas(args, sys.argv[1:]))
    if args.replica_selftest:
        args.steps = 10 if args.steps is None else args.steps
        run_replica_selftest(args)
    elif args.impl == "reference":
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
