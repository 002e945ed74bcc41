"""Seeded synthetic inputs: initial polarization fields and electrode masks.

This module holds only input generation -- a counter-based random generator,
initial-state recipes and boundary masks.  It contains none of the method's
arithmetic, so both the GPU path and the CPU oracle can be fed from it.

Random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) evaluated in
counter mode, element ``i`` of stream ``seed`` being the output for state
``seed + (i + 1) * golden_gamma``; a uniform double is ``(u >> 11) * 2**-53``.
Element order is component-major, then x fastest, then y, then z, matching
the (3, nz, ny, nx) array layout.

The workloads stand in for the paper's BiFeO3 film simulations (a
1056 x 1056 x 32 nm film at 1 nm spacing, dt = 0.005 in reduced units, short
circuit or open top surface, in-plane or tip electrodes; Section Results).
The BFO coefficients the paper uses are not available, so every workload uses
the dimensionless Landau set a1 = -1, a11 = 0.5, a12 = 0.8 (a fixed misfit
strain assumed folded in), g = 0.5, L = 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

NEUMANN, DIRICHLET = 0, 1


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the SplitMix64 stream ``seed``."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the counter-based stream."""
    return (splitmix64(seed, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class Workload:
    """One film: grid, coefficients, initial state, boundary masks, run length."""
    name: str
    nx: int
    ny: int
    nz: int
    P0: np.ndarray                       # (3, nz, ny, nx) float64
    type_lo: np.ndarray                  # (ny, nx) int8, 1 = Dirichlet electrode
    volt_lo: np.ndarray                  # (ny, nx) float64 volts
    type_hi: np.ndarray
    volt_hi: np.ndarray
    eps: np.ndarray | None = None        # (nz, ny, nx) or None for eps = 1
    dx: float = 1.0
    a1: float = -1.0
    a11: float = 0.5
    a12: float = 0.8
    g: float = 0.5
    L: float = 1.0
    dt: float = 0.01
    steps: int = 1
    rtol: float = 1e-12
    maxit: int = 20000
    precision: str = "fp64"              # "fp64" or "fp32"
    solver: str = "pcg"                  # "pcg" (Jacobi-PCG) or "mg" (multigrid-PCG)
    periodic_z: bool = False
    n_air: int = 0                       # top layers that are air (P = 0; eps from the eps field)
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def _faces(nx, ny):
    z8 = np.zeros((ny, nx), np.int8)
    zv = np.zeros((ny, nx), np.float64)
    return z8.copy(), zv.copy(), z8.copy(), zv.copy()


def random_film(nx, ny, nz, seed, lo=-0.01, hi=0.01, base=(0.0, 0.0, 0.0)) -> np.ndarray:
    """base + U[lo, hi) per component, component-major then x fastest."""
    n = nx * ny * nz
    u = uniform(seed, 3 * n).reshape(3, nz, ny, nx)
    P = lo + (hi - lo) * u
    for c in range(3):
        P[c] += base[c]
    return P


def stripe_film(nx, ny, nz, seed, width=16, noise=0.02) -> np.ndarray:
    """Stripes normal to [110] (stripe id = (x + y) // width), each stripe one of
    the four <111> variants (+-1, +-1, -1)/sqrt(3) drawn at random, plus
    U[-noise, noise) per component.  The variant draw uses stream seed + 1000."""
    variants = np.array([[1, 1, -1], [-1, 1, -1], [-1, -1, -1], [1, -1, -1]], np.float64) / np.sqrt(3.0)
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    sid = (x + y) // width                                   # (ny, nx)
    nstripes = int(sid.max()) + 1
    pick = np.minimum((uniform(seed + 1000, nstripes) * 4).astype(np.int64), 3)
    v = variants[pick[sid]]                                  # (ny, nx, 3)
    P = random_film(nx, ny, nz, seed, -noise, noise)
    for c in range(3):
        P[c] += v[None, :, :, c]
    return P


def grounded_both(nx, ny):
    tl, vl, th, vh = _faces(nx, ny)
    tl[:] = DIRICHLET
    th[:] = DIRICHLET
    return tl, vl, th, vh


def strip_electrodes(nx, ny, v=2.0):
    """Two strips spanning all y on the top face, width nx/8 and gap nx/4,
    at +v and -v (256-wide film: x in [64, 96) at +v, [160, 192) at -v).
    The rest of the top face and the whole bottom face are open (Neumann)."""
    tl, vl, th, vh = _faces(nx, ny)
    w = nx // 8
    a0, b0 = nx // 4, nx // 4 + w
    a1, b1 = b0 + nx // 4, b0 + nx // 4 + w
    th[:, a0:b0] = DIRICHLET
    vh[:, a0:b0] = +v
    th[:, a1:b1] = DIRICHLET
    vh[:, a1:b1] = -v
    return tl, vl, th, vh


def tip_electrode(nx, ny, v=3.0):
    """Grounded bottom; a centred square Dirichlet tip of side nx/8 at v on the
    top (1024-wide film: x, y in [448, 576)); the rest of the top open."""
    tl, vl, th, vh = _faces(nx, ny)
    tl[:] = DIRICHLET
    s = nx // 8
    x0, y0 = (nx - s) // 2, (ny - s) // 2
    th[y0:y0 + s, x0:x0 + s] = DIRICHLET
    vh[y0:y0 + s, x0:x0 + s] = v
    return tl, vl, th, vh


def film_fp64_grounded(nx=32, ny=32, nz=32, steps=200, seed=0) -> Workload:
    """Plain FP64 film between grounded electrodes, P ~ U[-0.01, 0.01]
    (32^3, 200 steps, dt 0.01, CG to 1e-12)."""
    P0 = random_film(nx, ny, nz, seed)
    tl, vl, th, vh = grounded_both(nx, ny)
    return Workload("fp64_grounded_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, P0, tl, vl, th, vh,
                    dt=0.01, steps=steps, rtol=1e-12, precision="fp64", solver="pcg", seed=seed)


def film_strip_fp32(nx=256, ny=256, nz=64, steps=5000, seed=1, v=2.0) -> Workload:
    """FP32 thin film poled +z with 1% noise, in-plane bias from two top strip
    electrodes at +-2 (256 x 256 x 64, 5000 steps, dt 0.01, CG to 1e-8)."""
    P0 = random_film(nx, ny, nz, seed, base=(0.0, 0.0, 1.0))
    tl, vl, th, vh = strip_electrodes(nx, ny, v)
    return Workload("fp32_strips_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, P0, tl, vl, th, vh,
                    dt=0.01, steps=steps, rtol=1e-8, precision="fp32", solver="pcg", seed=seed)


def film_tip_fp32(nx=1024, ny=1024, nz=128, steps=1000, seed=2, v=3.0) -> Workload:
    """Micron-scale FP32 film: 4-variant <111> stripe domains (period 32, 2%
    noise), grounded bottom, centred square tip electrode at 3.0 on top,
    multigrid-preconditioned CG to 1e-7 (1024 x 1024 x 128, 1000 steps, dt 0.005)."""
    P0 = stripe_film(nx, ny, nz, seed)
    tl, vl, th, vh = tip_electrode(nx, ny, v)
    return Workload("fp32_tip_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, P0, tl, vl, th, vh,
                    dt=0.005, steps=steps, rtol=1e-7, maxit=500, precision="fp32", solver="mg", seed=seed)


def film_adjoint_fp64(nx=128, ny=128, nz=32, steps=500, seed=3, v=2.0) -> Workload:
    """FP64 differentiation film: strip electrodes, +z poled with 1% noise."""
    P0 = random_film(nx, ny, nz, seed, base=(0.0, 0.0, 1.0))
    tl, vl, th, vh = strip_electrodes(nx, ny, v)
    return Workload("fp64_adjoint_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, P0, tl, vl, th, vh,
                    dt=0.01, steps=steps, rtol=1e-12, precision="fp64", solver="pcg", seed=seed)


# ------------------------------------------------------ batched hysteresis sweep

BATCH_SHAPES = ((32, 32, 32), (64, 64, 32), (96, 96, 48), (128, 128, 64))


def tri_wave(s):
    """Unit triangle wave of period 1: 0 at 0, 1 at 1/4, -1 at 3/4 (the shape of
    the electrode voltage ramps of a hysteresis sweep; an input schedule)."""
    f = np.asarray(s, dtype=np.float64)
    f = f - np.floor(f)
    return np.where(f < 0.25, 4.0 * f, np.where(f < 0.75, 2.0 - 4.0 * f, 4.0 * f - 4.0))


def ramp_volts(amplitude, period, step):
    """Electrode voltage during step `step` of a triangular ramp."""
    return float(amplitude * tri_wave(step / period))


def batch_draws(nfilms=64, seed=4, shapes=BATCH_SHAPES):
    """Per film: (grid shape, ramp amplitude A ~ U[1.5, 4.0], period T ~
    U[500, 2000] steps), from stream `seed` (three draws per film)."""
    u = uniform(seed, 3 * nfilms).reshape(nfilms, 3)
    return [(shapes[min(int(u[i, 0] * len(shapes)), len(shapes) - 1)], 1.5 + 2.5 * u[i, 1],
             500.0 + 1500.0 * u[i, 2]) for i in range(nfilms)]


def film_batch_hysteresis(nfilms=64, seed=4, steps=4000, shapes=BATCH_SHAPES, precision="fp32",
                          rtol=1e-6):
    """Independent films of a batched hysteresis sweep.  Film i: grid drawn
    uniformly from `shapes` (32^3, 64x64x32, 96x96x48, 128x128x64), the
    grounded-film physics (P ~ U[-0.01, 0.01], stream seed * 1000 + i), a
    grounded bottom electrode and a whole-face top electrode driven by the
    ramp V(s) = A tri(s / T) with A ~ U[1.5, 4.0] and T ~ U[500, 2000] steps
    (extra["ramp"] = (A, T)); dt 0.01, Jacobi-PCG to 1e-6.  The draws of
    stream `seed` are (shape, A, T) per film."""
    films = []
    for i, ((nx, ny, nz), amp, period) in enumerate(batch_draws(nfilms, seed, shapes)):
        fseed = seed * 1000 + i
        P0 = random_film(nx, ny, nz, fseed)
        tl, vl, th, vh = grounded_both(nx, ny)
        films.append(Workload("batch%d_%dx%dx%d" % (i, nx, ny, nz), nx, ny, nz, P0, tl, vl, th, vh,
                              dt=0.01, steps=steps, rtol=rtol, maxit=20000, precision=precision,
                              solver="pcg", seed=fseed, extra={"ramp": (amp, period)}))
    return films


def film_open_air(nx=64, ny=64, nz=37, n_air=5, steps=200, seed=5, precision="fp32", eps_film=100.0,
                  eps_air=1.0) -> Workload:
    """Open-circuit film with air on top (Section Results: a Neumann top surface
    over 5 layers of air, permittivity 1 in air against 100 in the film):
    4-variant <111> stripe domains (period 32, 2% noise) in the nz - n_air
    film layers, P = 0 in the air, grounded bottom electrode, open top.
    dt 0.005, Jacobi-PCG to 1e-8."""
    P0 = stripe_film(nx, ny, nz, seed)
    P0[:, nz - n_air:] = 0.0
    eps = np.full((nz, ny, nx), eps_film)
    eps[nz - n_air:] = eps_air
    tl, vl, th, vh = _faces(nx, ny)
    tl[:] = DIRICHLET
    return Workload("open_air_%dx%dx%d" % (nx, ny, nz), nx, ny, nz, P0, tl, vl, th, vh, eps=eps,
                    dt=0.005, steps=steps, rtol=1e-8, precision=precision, solver="pcg", n_air=n_air, seed=seed)
