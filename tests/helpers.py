"""Shared test helpers: run a workload through the oracle or the GPU library."""
import numpy as np

import oracle as O
from paper_1202_6116_gb300 import workloads as W


def oracle_grid(w: W.Workload) -> O.Grid:
    return O.Grid(w.nx, w.ny, w.nz, w.dx, w.periodic_z, w.type_lo, w.volt_lo, w.type_hi, w.volt_hi,
                  w.eps, w.n_air)


def oracle_params(w: W.Workload, rtol=None) -> O.Params:
    return O.Params(w.a1, w.a11, w.a12, w.g, w.L, w.dt, w.rtol if rtol is None else rtol, w.maxit)


def oracle_run(w: W.Workload, steps=None, rtol=None, phi0=None):
    P, phi, st, info = O.step(oracle_grid(w), oracle_params(w, rtol), w.P0, phi0,
                              w.steps if steps is None else steps)
    return P, phi, st, info


def relerr(a, b):
    """max|a - b| / max|b| (normwise, per field)."""
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def switched_fraction(P, threshold=0.3):
    """Fraction of cells whose P_x exceeds the threshold."""
    return float((P[0] > threshold).mean())


def mixed_workload(nx, ny, nz, seed, precision="fp64", eps=False, volts=True, steps=10, rtol=1e-12,
                   amp=0.5, tol_dirichlet=0.5):
    rng = np.random.default_rng(seed)
    tl = (rng.random((ny, nx)) < tol_dirichlet).astype(np.int8)
    th = (rng.random((ny, nx)) < tol_dirichlet).astype(np.int8)
    tl[0, 0] = 1
    vl = rng.uniform(-1, 1, (ny, nx)) if volts else np.zeros((ny, nx))
    vh = rng.uniform(-1, 1, (ny, nx)) if volts else np.zeros((ny, nx))
    e = rng.uniform(0.5, 3.0, (nz, ny, nx)) if eps else None
    P0 = W.random_film(nx, ny, nz, seed, -amp, amp)
    return W.Workload("mixed_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, P0, tl, vl, th, vh, eps=e,
                      steps=steps, rtol=rtol, precision=precision, seed=seed)
