"""Gradients of a TDGL trajectory through the library's discrete adjoint.

``trajectory(P0, coeffs, volt_lo, volt_hi, spec)`` runs ``spec.steps``
forward-Euler TDGL + Poisson steps (Eq. TDGL, Eqs. rho and Poisson, Section
Time Integration) and returns the final polarization.  It is a
``torch.autograd.Function``: the backward pass walks the steps in reverse
with ``pf_adjoint_step`` and returns dJ/dP0, dJ/d(a1, a11, a12, g) and the
gradients with respect to the two face-voltage maps.  States are
checkpointed every ``spec.checkpoint_every`` steps in the forward pass; the
backward pass recomputes each segment from its checkpoint (the forward step
is deterministic, so the recomputed states are bit-identical) and keeps only
that segment's states.

All arithmetic runs in the CUDA library; this module only moves tensors.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import pf
from .film import Film
from .workloads import Workload


@dataclass
class TrajectorySpec:
    workload: Workload          # grid, masks, dt, L, solver settings (P0, coefficients and volts are overridden)
    steps: int
    checkpoint_every: int = 50
    device: str = "cuda"


def _film(spec: TrajectorySpec, P0, coeffs, volt_lo, volt_hi) -> Film:
    c = [float(v) for v in coeffs.detach().cpu().double()]
    w = spec.workload.with_(a1=c[0], a11=c[1], a12=c[2], g=c[3],
                            volt_lo=volt_lo.detach().cpu().double().numpy(),
                            volt_hi=volt_hi.detach().cpu().double().numpy())
    # the paper's warm start (last potential): recomputed segments repeat the forward pass exactly
    return Film(w, device=spec.device, P0=P0, flags=pf.PF_FLAG_ADJOINT | pf.PF_FLAG_WARM_LAST)


class _Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, P0, coeffs, volt_lo, volt_hi, spec):
        film = _film(spec, P0, coeffs, volt_lo, volt_hi)
        K = max(1, int(spec.checkpoint_every))
        ckpts = []
        done = 0
        while done < spec.steps:
            n = min(K, spec.steps - done)
            ckpts.append((film.P.clone(), film.phi.clone(), n))
            film.step(n)
            done += n
        ctx.film, ctx.ckpts, ctx.spec = film, ckpts, spec
        ctx.in_meta = [(t.dtype, t.device) for t in (P0, coeffs, volt_lo, volt_hi)]
        return film.P.clone().to(P0.dtype)

    @staticmethod
    def backward(ctx, gP):
        film, spec = ctx.film, ctx.spec
        dev = film.P.device
        lam = gP.detach().to(device=dev, dtype=film.dtype).contiguous().clone()
        lam_out = torch.empty_like(lam)
        grad = torch.zeros(4, dtype=torch.float64, device=dev)
        gv = torch.zeros((2,) + tuple(film.w.type_lo.shape), dtype=torch.float64, device=dev)
        for P_c, phi_c, n in reversed(ctx.ckpts):
            film.P.copy_(P_c)
            film.phi.copy_(phi_c)
            states = [P_c]
            for _ in range(n - 1):
                film.step(1)
                states.append(film.P.clone())
            for k in range(n - 1, -1, -1):
                film.P.copy_(states[k])
                pf.pf_adjoint_step(film.ctx, lam, lam_out, grad, gv)
                lam, lam_out = lam_out, lam
        film.close()
        (tP, dP), (tc, dc), (tl, dl), (th, dh) = ctx.in_meta
        return (lam.to(dtype=tP, device=dP), grad.to(dtype=tc, device=dc), gv[0].to(dtype=tl, device=dl),
                gv[1].to(dtype=th, device=dh), None)


def trajectory(P0: torch.Tensor, coeffs: torch.Tensor, volt_lo: torch.Tensor, volt_hi: torch.Tensor,
               spec: TrajectorySpec) -> torch.Tensor:
    """Final polarization after spec.steps steps (differentiable in all four inputs).

    P0: (3, nz, ny, nx) device tensor; coeffs: (a1, a11, a12, g) as a float64
    tensor; volt_lo / volt_hi: (ny, nx) face-voltage maps (used where the
    workload's masks mark electrodes)."""
    return _Trajectory.apply(P0, coeffs, volt_lo, volt_hi, spec)


def final_state(spec: TrajectorySpec, coeffs, volt_lo, volt_hi, P0=None) -> torch.Tensor:
    """Forward pass only (no autograd bookkeeping), e.g. for finite differences."""
    w = spec.workload
    if P0 is None:
        P0 = torch.as_tensor(np.ascontiguousarray(w.P0), device=spec.device)
    film = _film(spec, P0, torch.as_tensor(coeffs, dtype=torch.float64),
                 torch.as_tensor(volt_lo, dtype=torch.float64), torch.as_tensor(volt_hi, dtype=torch.float64))
    try:
        film.step(spec.steps)
        return film.P.clone()
    finally:
        film.close()
