"""Autotuner of the fine-grid plane-march tiling (tile shape and z-block depth).

For a film shape it times every candidate tiling (``pf_set_tiling``: cells
per thread along x, which sets the tile width, z planes per tile, resident
blocks per SM) on a scratch copy of the film and keeps the fastest.  The
objective is device time per Krylov iteration (CUDA events on the film's
stream), so candidates are compared fairly even when the iteration counts of
the timed steps differ.  Results are cached per (shape, precision, solver,
permittivity) in memory and, optionally, in a JSON file.
"""
from __future__ import annotations

import json
import os

import torch

from . import pf
from .film import Film
from .workloads import Workload

_CACHE: dict = {}


def key_of(w: Workload) -> str:
    return "%dx%dx%d/%s/%s/%s" % (w.nx, w.ny, w.nz, w.precision, w.solver, "eps" if w.eps is not None else "unit")


def candidates(w: Workload, tz_list=(1, 2, 4, 8, 16, 32), bps_list=(0, 2)):
    """Valid (vx, tz, blocks_per_sm) triples for this film.  vx: 16 bytes of
    cells per thread (4 FP32 / 2 FP64; needs nx divisible) or one cell, i.e.
    tiles of 64 x 16 / 32 x 16 or 16 x 16 columns; tz up to nz."""
    vmax = 4 if w.precision == "fp32" else 2
    vxs = [vmax, 1] if w.nx % vmax == 0 else [1]
    tzs = sorted({min(t, w.nz) for t in tz_list})
    out = []
    for vx in vxs:
        for tz in tzs:
            for bps in bps_list:
                out.append((vx, tz, bps))
    return out


def time_tiling(f: Film, tiling, steps: int, warmup: int) -> float:
    """Device ms per Krylov iteration of `steps` steps under this tiling."""
    pf.pf_set_tiling(f.ctx, *tiling)
    f.step(warmup, ok=(pf.PF_OK, pf.PF_ERR_NOCONV))
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(f.stream)
    _, info = f.step(steps, ok=(pf.PF_OK, pf.PF_ERR_NOCONV))
    b.record(f.stream)
    b.synchronize()
    return a.elapsed_time(b) / max(1, info["total_iters"] + steps)


def tune(w: Workload, steps: int = 3, warmup: int = 1, cache_file: str | None = None, device="cuda") -> dict:
    """Best tiling for films shaped like w: {"vx", "tz", "blocks_per_sm",
    "ms_per_iter", "default_ms_per_iter", "table"}.  Runs on a scratch film."""
    key = key_of(w)
    if key in _CACHE:
        return _CACHE[key]
    if cache_file and os.path.exists(cache_file):
        with open(cache_file) as fh:
            disk = json.load(fh)
        if key in disk:
            _CACHE[key] = disk[key]
            return disk[key]
    f = Film(w, device=device)
    try:
        d = pf.pf_get_tiling(f.ctx)
        default = (d.vx, d.tz, d.blocks_per_sm)
        P0, phi0 = f.P.clone(), f.phi.clone()
        table = []
        for t in [default] + [c for c in candidates(w) if c != default]:
            f.P.copy_(P0)
            f.phi.copy_(phi0)
            table.append((t, time_tiling(f, t, steps, warmup)))
        best, ms = min(table, key=lambda e: e[1])
        res = {"vx": best[0], "tz": best[1], "blocks_per_sm": best[2], "ms_per_iter": ms,
               "default": list(default), "default_ms_per_iter": table[0][1],
               "table": [[list(t), m] for t, m in table]}
    finally:
        f.close()
    _CACHE[key] = res
    if cache_file:
        disk = {}
        if os.path.exists(cache_file):
            with open(cache_file) as fh:
                disk = json.load(fh)
        disk[key] = res
        with open(cache_file, "w") as fh:
            json.dump(disk, fh, indent=1)
    return res


def apply(f: Film, res: dict):
    """Set a tuned tiling on a film."""
    pf.pf_set_tiling(f.ctx, res["vx"], res["tz"], res["blocks_per_sm"])
