"""ctypes view of the plain FP64 C oracle (``pf_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The GPU library never
imports this package and this package never imports the GPU library.

Arrays are numpy float64 (int8 for boundary masks); P is (3, nz, ny, nx),
scalar fields are (nz, ny, nx), face masks are (ny, nx).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double),
                ("periodic_z", C.c_int),
                ("type_lo", C.c_void_p), ("volt_lo", C.c_void_p),
                ("type_hi", C.c_void_p), ("volt_hi", C.c_void_p),
                ("eps", C.c_void_p), ("n_air", C.c_int)]


class _Params(C.Structure):
    _fields_ = [("a1", C.c_double), ("a11", C.c_double), ("a12", C.c_double),
                ("g", C.c_double), ("L", C.c_double), ("dt", C.c_double),
                ("rtol", C.c_double), ("maxit", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("steps_done", C.c_int), ("last_iters", C.c_int), ("total_iters", C.c_long),
                ("last_relres", C.c_double), ("nonconverged", C.c_int)]


_libs = {}
_openmp = False


def lib():
    """The loaded oracle library: the serial build, or the OpenMP build of the
    same source inside ``openmp()`` (timing baselines only)."""
    global _lib
    key = "omp" if _openmp else "serial"
    if key not in _libs:
        path = _build.build(openmp=_openmp)
        L = C.CDLL(path)
        vp, d, i, l = C.c_void_p, C.c_double, C.c_int, C.c_long
        L.or_landau_energy.restype = d
        L.or_landau_energy.argtypes = [vp, l, d, d, d]
        L.or_landau_force.argtypes = [vp, l, d, d, d, vp]
        for f in (L.or_laplacian, L.or_rhs, L.or_apply, L.or_field):
            f.argtypes = [vp, vp, vp]
        L.or_diag.argtypes = [vp, vp]
        L.or_has_dirichlet.argtypes = [vp]
        L.or_solve.argtypes = [vp, vp, vp, d, i, vp, vp]
        L.or_solve_potential.argtypes = [vp, vp, vp, d, i, vp, vp]
        L.or_step.argtypes = [vp, vp, vp, vp, i, vp]
        L.or_rate.argtypes = [vp, vp, vp, vp, vp]
        L.or_rate_at.argtypes = [vp, vp, vp, vp, vp, i, vp]
        L.or_step_ex.argtypes = [vp, vp, i, i, l, vp, vp, i, d, C.c_ulonglong, vp]
        L.or_philox.argtypes = [C.c_ulonglong, C.c_ulonglong, C.c_ulonglong, vp]
        L.or_gauss4.argtypes = [C.c_ulonglong, C.c_ulonglong, C.c_ulonglong, vp]
        L.or_energy.restype = d
        L.or_energy.argtypes = [vp, vp, vp, d]
        L.or_adjoint_step.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.or_diagnostics.argtypes = [vp, vp, vp, vp, d, vp]
        L.or_threads.restype = i
        L.or_threads.argtypes = []
        _libs[key] = L
    _lib = _libs[key]
    return _lib


class openmp:
    """Context in which the oracle functions run the OpenMP build (all host
    cores, OMP_NUM_THREADS permitting).  For timing baselines only: the
    tests use the serial build."""

    def __enter__(self):
        global _openmp
        self._prev = _openmp
        _openmp = True
        return self

    def __exit__(self, *exc):
        global _openmp
        _openmp = self._prev
        return False


def threads() -> int:
    """Threads the current build's loops run on (1 for the serial build)."""
    return int(lib().or_threads())


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


@dataclass
class Grid:
    """Grid, boundary masks and permittivity (the oracle's own description)."""
    nx: int
    ny: int
    nz: int
    dx: float = 1.0
    periodic_z: bool = False
    type_lo: np.ndarray | None = None
    volt_lo: np.ndarray | None = None
    type_hi: np.ndarray | None = None
    volt_hi: np.ndarray | None = None
    eps: np.ndarray | None = None
    n_air: int = 0                      # top layers that are air (P = 0, no wall energy across)

    def __post_init__(self):
        m = (self.ny, self.nx)
        def mask(a):
            return np.zeros(m, np.int8) if a is None else np.ascontiguousarray(a, np.int8).reshape(m)
        def volt(a):
            return np.zeros(m) if a is None else _f64(a).reshape(m)
        self.type_lo, self.type_hi = mask(self.type_lo), mask(self.type_hi)
        self.volt_lo, self.volt_hi = volt(self.volt_lo), volt(self.volt_hi)
        if self.eps is not None:
            self.eps = _f64(self.eps).reshape(self.shape)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    def _c(self):
        g = _Grid(self.nx, self.ny, self.nz, float(self.dx), int(bool(self.periodic_z)),
                  _ptr(self.type_lo), _ptr(self.volt_lo), _ptr(self.type_hi), _ptr(self.volt_hi),
                  _ptr(self.eps), int(self.n_air))
        return g


@dataclass
class Params:
    a1: float = -1.0
    a11: float = 0.5
    a12: float = 0.8
    g: float = 0.5
    L: float = 1.0
    dt: float = 0.01
    rtol: float = 1e-12
    maxit: int = 100000

    def _c(self):
        return _Params(self.a1, self.a11, self.a12, self.g, self.L, self.dt, self.rtol, int(self.maxit))


def landau_energy(P, prm: Params) -> float:
    P = _f64(P)
    n = P.size // 3
    return lib().or_landau_energy(_ptr(P), n, prm.a1, prm.a11, prm.a12)


def landau_force(P, prm: Params):
    P = _f64(P)
    out = np.empty_like(P)
    lib().or_landau_force(_ptr(P), P.size // 3, prm.a1, prm.a11, prm.a12, _ptr(out))
    return out


def _unary(fn, G: Grid, a, out_shape):
    a = _f64(a)
    out = np.empty(out_shape)
    g = G._c()
    fn(C.byref(g), _ptr(a), _ptr(out))
    return out


def laplacian(G: Grid, f):
    return _unary(lib().or_laplacian, G, _f64(f).reshape(G.shape), G.shape)


def rhs(G: Grid, P):
    return _unary(lib().or_rhs, G, _f64(P).reshape((3,) + G.shape), G.shape)


def apply(G: Grid, phi):
    return _unary(lib().or_apply, G, _f64(phi).reshape(G.shape), G.shape)


def field(G: Grid, phi):
    return _unary(lib().or_field, G, _f64(phi).reshape(G.shape), (3,) + G.shape)


def diag(G: Grid):
    out = np.empty(G.shape)
    g = G._c()
    lib().or_diag(C.byref(g), _ptr(out))
    return out


def has_dirichlet(G: Grid) -> bool:
    g = G._c()
    return bool(lib().or_has_dirichlet(C.byref(g)))


def solve(G: Grid, b, phi0=None, rtol=1e-14, maxit=100000):
    """Jacobi-PCG solve of A phi = b.  Returns (phi, status, iters, relres)."""
    b = _f64(b).reshape(G.shape)
    phi = np.zeros(G.shape) if phi0 is None else _f64(phi0).reshape(G.shape).copy()
    it, rel = C.c_int(0), C.c_double(0.0)
    g = G._c()
    st = lib().or_solve(C.byref(g), _ptr(b), _ptr(phi), float(rtol), int(maxit),
                        C.byref(it), C.byref(rel))
    return phi, st, it.value, rel.value


def solve_potential(G: Grid, P, phi0=None, rtol=1e-14, maxit=100000):
    P = _f64(P).reshape((3,) + G.shape)
    phi = np.zeros(G.shape) if phi0 is None else _f64(phi0).reshape(G.shape).copy()
    it, rel = C.c_int(0), C.c_double(0.0)
    g = G._c()
    st = lib().or_solve_potential(C.byref(g), _ptr(P), _ptr(phi), float(rtol), int(maxit),
                                  C.byref(it), C.byref(rel))
    return phi, st, it.value, rel.value


def step(G: Grid, prm: Params, P, phi=None, nsteps=1):
    """nsteps forward-Euler steps.  Returns (P, phi, status, info dict)."""
    P = _f64(P).reshape((3,) + G.shape).copy()
    phi = np.zeros(G.shape) if phi is None else _f64(phi).reshape(G.shape).copy()
    info = _Info()
    g, p = G._c(), prm._c()
    st = lib().or_step(C.byref(g), C.byref(p), _ptr(P), _ptr(phi), int(nsteps), C.byref(info))
    d = dict(steps_done=info.steps_done, last_iters=info.last_iters,
             total_iters=info.total_iters, last_relres=info.last_relres,
             nonconverged=info.nonconverged)
    return P, phi, st, d


INTEGRATORS = {"euler": 0, "heun": 1}


def rate(G: Grid, prm: Params, P, phi):
    """TDGL rate L(-df/dP + g Lap P + E(phi)) at state P with potential phi."""
    P = _f64(P).reshape((3,) + G.shape)
    phi = _f64(phi).reshape(G.shape)
    out = np.empty_like(P)
    g, p = G._c(), prm._c()
    lib().or_rate(C.byref(g), C.byref(p), _ptr(P), _ptr(phi), _ptr(out))
    return out


def rate_at(G: Grid, prm: Params, P, phi, cells):
    """TDGL rate at the listed linear cell indices: array (len(cells), 3)."""
    P = _f64(P).reshape((3,) + G.shape)
    phi = _f64(phi).reshape(G.shape)
    idx = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.empty((len(idx), 3))
    g, p = G._c(), prm._c()
    lib().or_rate_at(C.byref(g), C.byref(p), _ptr(P), _ptr(phi), _ptr(idx), len(idx), _ptr(out))
    return out


def step_ex(G: Grid, prm: Params, P, phi=None, nsteps=1, integrator="euler", every=1, n0=0, sigma=0.0, seed=0):
    """nsteps steps of forward Euler or of the paper's predictor-corrector
    ("heun"), the potential solved only on global steps n0 + s that are
    multiples of every; sigma > 0 adds the thermal random force (sigma
    sqrt(dt) standard normal draws per cell, component and step).  Returns
    (P, phi, status, info dict)."""
    P = _f64(P).reshape((3,) + G.shape).copy()
    phi = np.zeros(G.shape) if phi is None else _f64(phi).reshape(G.shape).copy()
    info = _Info()
    g, p = G._c(), prm._c()
    st = lib().or_step_ex(C.byref(g), C.byref(p), INTEGRATORS[integrator], int(every), int(n0), _ptr(P),
                          _ptr(phi), int(nsteps), float(sigma), int(seed), C.byref(info))
    d = dict(steps_done=info.steps_done, last_iters=info.last_iters,
             total_iters=info.total_iters, last_relres=info.last_relres,
             nonconverged=info.nonconverged)
    return P, phi, st, d


def philox(seed, step, cell):
    """The four 32-bit Philox4x32-10 words for counter (cell, step), key seed."""
    out = (C.c_uint * 4)()
    lib().or_philox(int(seed), int(step), int(cell), C.cast(out, C.c_void_p))
    return list(out)


def gauss4(seed, step, cell):
    """Four standard normal variates (Box-Muller of the Philox words)."""
    out = np.zeros(4)
    lib().or_gauss4(int(seed), int(step), int(cell), _ptr(out))
    return out


def energy(G: Grid, prm: Params, P, rtol=1e-14) -> float:
    P = _f64(P).reshape((3,) + G.shape)
    g, p = G._c(), prm._c()
    return lib().or_energy(C.byref(g), C.byref(p), _ptr(P), float(rtol))


def adjoint_step(G: Grid, prm: Params, P, lam, psi=None):
    """Transposed Jacobian of one forward step at state P applied to lam.

    Returns (lam_out, psi, grad[4] (a1, a11, a12, g), gv_lo, gv_hi, status,
    iters): the step's sensitivities alone (not accumulated)."""
    P = _f64(P).reshape((3,) + G.shape)
    lam = _f64(lam).reshape((3,) + G.shape)
    out = np.empty_like(lam)
    psi = np.zeros(G.shape) if psi is None else _f64(psi).reshape(G.shape).copy()
    grad = np.zeros(4)
    gv_lo = np.zeros((G.ny, G.nx))
    gv_hi = np.zeros((G.ny, G.nx))
    it = C.c_int(0)
    g, p = G._c(), prm._c()
    st = lib().or_adjoint_step(C.byref(g), C.byref(p), _ptr(P), _ptr(lam), _ptr(out), _ptr(psi),
                               _ptr(grad), _ptr(gv_lo), _ptr(gv_hi), C.byref(it))
    return out, psi, grad, gv_lo, gv_hi, st, it.value


def gradient(G: Grid, prm: Params, P0, lam_final, nsteps, phi0=None):
    """Reverse pass over nsteps forward steps from (P0, phi0): every state is
    kept, then the adjoint steps run backwards from lam_final = dJ/dP_nsteps.
    Returns (dJ/dP0, dJ/d(a1, a11, a12, g), dJ/dvolt_lo, dJ/dvolt_hi)."""
    states = [_f64(P0).reshape((3,) + G.shape).copy()]
    phi = None if phi0 is None else _f64(phi0)
    for _ in range(nsteps):
        P, phi, st, _info = step(G, prm, states[-1], phi, 1)
        assert st == OK
        states.append(P)
    lam = _f64(lam_final).reshape((3,) + G.shape).copy()
    grad = np.zeros(4)
    gv_lo = np.zeros((G.ny, G.nx))
    gv_hi = np.zeros((G.ny, G.nx))
    psi = None
    for k in range(nsteps - 1, -1, -1):
        lam, psi, gk, glo, ghi, st, _it = adjoint_step(G, prm, states[k], lam, psi)
        assert st == OK
        grad += gk
        gv_lo += glo
        gv_hi += ghi
    return lam, grad, gv_lo, gv_hi


DIAG_NAMES = ("mean_px", "mean_py", "mean_pz", "switched_fraction", "f_landau", "f_grad", "f_elec")


def diagnostics(G: Grid, prm: Params, P, phi, threshold=0.3) -> dict:
    """Mean P, switched fraction (P_x > threshold) and the three energy terms."""
    P = _f64(P).reshape((3,) + G.shape)
    phi = _f64(phi).reshape(G.shape)
    out = np.zeros(7)
    g, p = G._c(), prm._c()
    lib().or_diagnostics(C.byref(g), C.byref(p), _ptr(P), _ptr(phi), float(threshold), _ptr(out))
    return dict(zip(DIAG_NAMES, out.tolist()))


OK, NOCONV = 0, 3
