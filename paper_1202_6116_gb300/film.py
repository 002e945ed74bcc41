"""A film simulation held in torch device tensors, driven through the C ABI.

PyTorch supplies device memory and the stream; every computation runs in the
CUDA library through ``pf.py``.
"""
from __future__ import annotations

import numpy as np
import torch

from . import pf
from .workloads import Workload


def make_params(w: Workload, **overrides) -> pf.pf_params:
    p = pf.pf_params()
    p.nx, p.ny, p.nz, p.dx = w.nx, w.ny, w.nz, w.dx
    p.a1, p.a11, p.a12, p.g, p.L, p.dt = w.a1, w.a11, w.a12, w.g, w.L, w.dt
    p.precision = pf.PF_FP32 if w.precision == "fp32" else pf.PF_FP64
    p.solver = pf.PF_PCG_MG if w.solver == "mg" else pf.PF_PCG_JACOBI
    p.poisson_rtol = w.rtol
    p.poisson_maxit = w.maxit
    p.periodic_z = int(bool(w.periodic_z))
    p.has_eps = int(w.eps is not None)
    p.n_air = int(w.n_air)
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class Film:
    """Device state (P, phi, eps, workspace) of one film plus its context."""

    def __init__(self, w: Workload, device="cuda", stream=None, phi0=None, P0=None, **overrides):
        """P0 (optional): a device tensor that replaces w.P0 (copied)."""
        self.w = w
        self.params = make_params(w, **overrides)
        self.dtype = torch.float32 if self.params.precision == pf.PF_FP32 else torch.float64
        dev = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        if P0 is not None:
            self.P = P0.detach().to(device=dev, dtype=self.dtype).clone().contiguous()
        else:
            self.P = torch.as_tensor(np.ascontiguousarray(w.P0), dtype=self.dtype, device=dev).contiguous()
        self.phi = torch.zeros(w.shape, dtype=self.dtype, device=dev) if phi0 is None else \
            torch.as_tensor(np.ascontiguousarray(phi0), dtype=self.dtype, device=dev).contiguous()
        self.eps = None if w.eps is None else \
            torch.as_tensor(np.ascontiguousarray(w.eps), dtype=self.dtype, device=dev).contiguous()
        nbytes = pf.pf_workspace_bytes(self.params)
        if nbytes == 0:
            raise ValueError("invalid parameters for this workload")
        self.ws_bytes = nbytes
        # torch's caching allocator returns 512-byte aligned blocks
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.ctx = pf.pf_create(self.params, self.stream.cuda_stream)
        pf.pf_bind(self.ctx, self.P, self.phi, self.eps, self.workspace, nbytes)
        self.set_bc(pf.PF_ZLO, w.type_lo, w.volt_lo)
        self.set_bc(pf.PF_ZHI, w.type_hi, w.volt_hi)

    def set_bc(self, face, types, volts):
        t = np.ascontiguousarray(types, dtype=np.int8).reshape(-1)
        v = np.ascontiguousarray(volts, dtype=np.float64).reshape(-1)
        pf.pf_set_bc(self.ctx, face, t, v)

    def set_noise(self, sigma, seed=0):
        """Thermal random force of the TDGL equation (sigma = 0: off)."""
        pf.pf_set_noise(self.ctx, sigma, seed)

    def step(self, nsteps=1, ok=(pf.PF_OK,)):
        st, info = pf.pf_step(self.ctx, nsteps, ok)
        return st, info.as_dict()

    def step_async(self, nsteps=1):
        """Enqueue steps without waiting (see pf_step_async); wait() reports them."""
        pf.pf_step_async(self.ctx, nsteps)

    def wait(self, ok=(pf.PF_OK,)):
        st, info = pf.pf_step_wait(self.ctx, ok)
        return st, info.as_dict()

    def true_residual(self, P=None):
        """FP64 (||b(P) - A phi||, ||b(P)||, ||b(P) - A phi_c||) of the bound
        potential and of the compensated one."""
        return pf.pf_true_residual(self.ctx, P)

    def solve_potential(self, ok=(pf.PF_OK,)):
        st, info = pf.pf_solve_potential(self.ctx, ok)
        return st, info.as_dict()

    def diagnostics(self, threshold=0.3):
        """Mean P, switched fraction and energy terms of the current state."""
        return pf.pf_diagnostics(self.ctx, threshold)

    def numpy(self):
        return (self.P.double().cpu().numpy(), self.phi.double().cpu().numpy())

    def close(self):
        if getattr(self, "ctx", None):
            pf.pf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
