"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each check is a closed form, an
exact discrete identity with an independent derivation, a library routine
(numpy dense LU) or a physical limit.  They are chosen so that a dropped term,
a wrong sign or factor, or a transposed operand in any oracle function fails
at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1202_6116_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def mixed_grid(nx, ny, nz, seed, eps=False, volts=False):
    rng = np.random.default_rng(seed)
    tl = (rng.random((ny, nx)) < 0.5).astype(np.int8)
    th = (rng.random((ny, nx)) < 0.5).astype(np.int8)
    tl[0, 0] = 1  # at least one electrode: A nonsingular
    vl = rng.uniform(-1, 1, (ny, nx)) if volts else np.zeros((ny, nx))
    vh = rng.uniform(-1, 1, (ny, nx)) if volts else np.zeros((ny, nx))
    e = rng.uniform(0.5, 3.0, (nz, ny, nx)) if eps else None
    return O.Grid(nx, ny, nz, 1.0, False, tl, vl, th, vh, e)


def uniform_field(G, vec):
    P = np.zeros((3,) + G.shape)
    for c in range(3):
        P[c] = vec[c]
    return P


# --------------------------------------------------------------- Landau (Eq. F_bulk)

def test_landau_minima_closed_form():
    g = json.load(open(os.path.join(GOLDEN, "landau_minima.json")))
    prm = O.Params(a1=g["a1"], a11=g["a11"], a12=g["a12"])
    for key, direction in (("T_001", (0, 0, 1)), ("O_110", (1, 1, 0)), ("R_111", (1, 1, 1))):
        p = math.sqrt(g[key]["p2"])
        P = np.array(direction, float).reshape(3, 1) * p
        f = O.landau_energy(P, prm)
        assert abs(f - g[key]["f"]) < 1e-14, key
        force = O.landau_force(P, prm)
        assert np.abs(force).max() < 1e-14, key            # stationary point
        # a stationary point along the ray: perturbing |P| raises f
        for s in (0.99, 1.01):
            assert O.landau_energy(P * s, prm) > f
    # R [111] is the global minimum for a12 < 2 a11: no random direction beats it
    rng = np.random.default_rng(0)
    d = rng.normal(size=(3, 2000))
    d /= np.linalg.norm(d, axis=0)
    best = np.inf
    for amp in np.linspace(0.3, 1.3, 41):
        P = d * amp
        e = np.array([O.landau_energy(P[:, i:i + 1], prm) for i in range(0, 2000, 50)])
        best = min(best, e.min())
    assert best > g["R_111"]["f"] - 1e-12


def test_landau_force_is_energy_gradient():
    prm = O.Params(a1=-1.3, a11=0.7, a12=0.45)
    rng = np.random.default_rng(1)
    P = rng.uniform(-1, 1, (3, 5))
    force = O.landau_force(P, prm)
    h = 1e-6
    for c in range(3):
        for i in range(5):
            Pp, Pm = P.copy(), P.copy()
            Pp[c, i] += h
            Pm[c, i] -= h
            fd = (O.landau_energy(Pp, prm) - O.landau_energy(Pm, prm)) / (2 * h)
            assert abs(fd - force[c, i]) < 1e-8


# ------------------------------------------------- homogeneous dynamics (Eq. TDGL)

@pytest.mark.parametrize("direction,coef", [((1, 1, 1), 5.2), ((0, 0, 1), 2.0), ((1, 1, 0), 3.6)])
def test_homogeneous_recurrence(direction, coef):
    """Uniform P between grounded electrodes carries no charge (phi = 0), so each
    nonzero component follows p <- p + dt (2 p - coef p^3) exactly, with coef =
    4 a11 + 2 a12 (#nonzero - 1) from Eq. F_bulk."""
    G = O.Grid(6, 5, 4, type_lo=np.ones((5, 6)), type_hi=np.ones((5, 6)))
    prm = O.Params(dt=0.01, rtol=1e-14)
    p0 = 0.1
    P0 = uniform_field(G, [p0 * d for d in direction])
    P, phi, st, info = O.step(G, prm, P0, None, 50)
    p = p0
    for _ in range(50):
        p = p + 0.01 * (2 * p - coef * p ** 3)
    for c in range(3):
        assert np.abs(P[c] - p * direction[c]).max() < 1e-15
    assert np.abs(phi).max() == 0.0
    assert info["total_iters"] == 0


def test_homogeneous_continuum_limit():
    """u = p^2 obeys the logistic law u' = 4u (1 - u/u_inf), u_inf = 1/2.6; forward
    Euler converges to it at first order."""
    G = O.Grid(2, 2, 2, periodic_z=True)
    uinf, u0, T = 1.0 / 2.6, 0.01, 2.0
    exact = uinf / (1 + (uinf / u0 - 1) * math.exp(-4 * T))
    errs = []
    for dt in (0.02, 0.01, 0.005):
        prm = O.Params(dt=dt)
        P, _, _, _ = O.step(G, prm, uniform_field(G, [math.sqrt(u0)] * 3), None, int(round(T / dt)))
        errs.append(abs(P[0, 0, 0, 0] ** 2 - exact))
    assert errs[0] / errs[1] == pytest.approx(2.0, rel=0.1)
    assert errs[1] / errs[2] == pytest.approx(2.0, rel=0.1)


# ---------------------------------------------- electrostatics (Eqs. rho, Poisson)

def test_short_circuit_uniform_film_has_no_field():
    G = O.Grid(5, 4, 6, type_lo=np.ones((4, 5)), type_hi=np.ones((4, 5)))
    P = uniform_field(G, [0.3, -0.2, 0.7])
    assert np.abs(O.rhs(G, P)).max() == 0.0
    phi, st, it, _ = O.solve_potential(G, P)
    assert np.abs(O.field(G, phi)).max() == 0.0


@pytest.mark.parametrize("eps", [1.0, 4.0])
def test_open_film_depolarizing_field(eps):
    """Uniform P_z in a film with open (Neumann) top and bottom: Gauss's law gives
    E_z = -P_z/eps inside the film (the bound surface charges are kept)."""
    nz = 10
    G = O.Grid(3, 3, nz, eps=np.full((nz, 3, 3), eps))
    P = uniform_field(G, [0.0, 0.0, 0.6])
    phi, st, it, _ = O.solve_potential(G, P)
    E = O.field(G, phi)
    assert np.abs(E[2, 1:-1] + 0.6 / eps).max() < 1e-12
    assert np.abs(E[:2]).max() < 1e-12
    assert abs(phi.mean()) < 1e-13                       # zero-mean gauge of the singular case


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("m", [1, 3])
def test_periodic_fourier_mode(axis, m):
    """P_axis = A sin(k s) on a fully periodic box: the discrete potential is
    phi = -(A/2) cot(k/2) cos(k s) (derived by hand from the face-mean divergence
    and the compact Laplacian); its continuum limit is -A cos(k s)/k."""
    n = 16
    G = O.Grid(n, n, n, periodic_z=True)
    k = 2 * math.pi * m / n
    s = np.arange(n)
    shape = [1, 1, 1]
    shape[2 - axis] = n
    A = 0.37
    P = np.zeros((3, n, n, n))
    P[axis] = (A * np.sin(k * s)).reshape(shape)
    phi, st, it, _ = O.solve_potential(G, P, rtol=1e-14)
    ref = (-(A / 2) / math.tan(k / 2) * np.cos(k * s)).reshape(shape) * np.ones((n, n, n))
    assert np.abs(phi - ref).max() < 1e-12
    if m == 1:
        cont = (-A * np.cos(k * s) / k).reshape(shape)
        assert np.abs(phi - cont).max() / np.abs(cont).max() < k * k / 12 * 1.01


@pytest.mark.parametrize("kind", ["DD", "NN", "DN"])
def test_z_eigenmodes(kind):
    """Closed-form eigenvectors of the z operator with x,y Fourier factors:
    DD  sin(pi m (z+1/2)/nz),          lambda_z = 4 sin^2(pi m/(2 nz))
    NN  cos(pi m (z+1/2)/nz),          lambda_z = 4 sin^2(pi m/(2 nz))
    DN  sin(pi (2m+1)(z+1/2)/(2 nz)),  lambda_z = 4 sin^2(pi (2m+1)/(4 nz))
    times cos(2 pi kx x/nx): lambda += 4 sin^2(pi kx/nx)."""
    nx, ny, nz = 8, 6, 7
    one = np.ones((ny, nx), np.int8)
    zero = np.zeros((ny, nx), np.int8)
    tl, th = {"DD": (one, one), "NN": (zero, zero), "DN": (one, zero)}[kind]
    G = O.Grid(nx, ny, nz, type_lo=tl, type_hi=th)
    z = np.arange(nz) + 0.5
    x = np.arange(nx)
    for m, kx in ((1, 0), (2, 1), (3, 3)):
        if kind == "DD":
            fz, lz = np.sin(math.pi * m * z / nz), 4 * math.sin(math.pi * m / (2 * nz)) ** 2
        elif kind == "NN":
            fz, lz = np.cos(math.pi * m * z / nz), 4 * math.sin(math.pi * m / (2 * nz)) ** 2
        else:
            fz, lz = (np.sin(math.pi * (2 * m + 1) * z / (2 * nz)),
                      4 * math.sin(math.pi * (2 * m + 1) / (4 * nz)) ** 2)
        lam = lz + 4 * math.sin(math.pi * kx / nx) ** 2
        v = fz[:, None, None] * np.cos(2 * math.pi * kx * x / nx)[None, None, :] * np.ones((nz, ny, nx))
        Av = O.apply(G, v)
        assert np.abs(Av - lam * v).max() < 1e-13
        if kind != "NN":
            phi, st, it, _ = O.solve(G, v, rtol=1e-14)
            assert np.abs(phi - v / lam).max() < 1e-12 * max(1.0, 1 / lam)


def test_series_capacitor_layers():
    """Layered eps(z) between a grounded bottom and a top electrode at V, P = 0:
    the displacement flux is uniform and each cell is two half-cells in series,
    so phi at cell k = V (sum_{j<k} 1/eps_j + 1/(2 eps_k)) / sum_j 1/eps_j."""
    nz = 9
    rng = np.random.default_rng(3)
    ez = rng.uniform(0.5, 20.0, nz)
    eps = ez[:, None, None] * np.ones((nz, 3, 4))
    V = 1.7
    G = O.Grid(4, 3, nz, type_lo=np.ones((3, 4)), type_hi=np.ones((3, 4)),
               volt_hi=np.full((3, 4), V), eps=eps)
    phi, st, it, _ = O.solve_potential(G, np.zeros((3, nz, 3, 4)), rtol=1e-14)
    inv = 1.0 / ez
    ref = V * (np.concatenate([[0.0], np.cumsum(inv)[:-1]]) + 0.5 * inv) / inv.sum()
    assert np.abs(phi[:, 1, 2] - ref).max() < 1e-12
    assert np.abs(phi - phi[:, :1, :1]).max() < 1e-13


def test_dense_bruteforce_ragged():
    """Dense operator of a ragged 6x5x4 grid with random masks and permittivity:
    symmetric positive definite; CG agrees with numpy's dense LU solve."""
    G = mixed_grid(6, 5, 4, seed=7, eps=True, volts=True)
    n = G.n
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = O.apply(G, e).ravel()
    assert np.abs(A - A.T).max() < 1e-14
    assert np.linalg.eigvalsh(A).min() > 1e-3
    assert np.allclose(np.diag(A), O.diag(G).ravel(), rtol=0, atol=1e-14)
    rng = np.random.default_rng(2)
    P = rng.uniform(-1, 1, (3,) + G.shape)
    b = O.rhs(G, P).ravel()
    ref = np.linalg.solve(A, b)
    phi, st, it, rel = O.solve(G, b, rtol=1e-14)
    assert st == O.OK
    assert np.abs(phi.ravel() - ref).max() / np.abs(ref).max() < 1e-12
    # warm start from a nearby guess gives the same answer
    phi2, st2, it2, _ = O.solve(G, b, phi0=ref.reshape(G.shape) * 1.01, rtol=1e-14)
    assert np.abs(phi2.ravel() - ref).max() / np.abs(ref).max() < 1e-12


def test_divergence_gradient_pairing():
    """With the face-value rules, grad = -div^T exactly (summation by parts with
    every boundary term cancelled): sum phi b(P) = -sum P . E(phi) at V = 0."""
    G = mixed_grid(7, 6, 5, seed=11, eps=True)
    rng = np.random.default_rng(5)
    for _ in range(3):
        P = rng.normal(size=(3,) + G.shape)
        phi = rng.normal(size=G.shape)
        lhs = np.sum(phi * O.rhs(G, P))
        rhs_ = -np.sum(P * O.field(G, phi))
        assert abs(lhs - rhs_) < 1e-11 * (1 + abs(lhs))


def test_laplacian_closed_forms():
    G = O.Grid(5, 4, 9)
    z = np.arange(9, dtype=float)[:, None, None] * np.ones((9, 4, 5))
    # quadratic: exact second difference 2 in the interior
    lap = O.laplacian(G, z ** 2)
    assert np.abs(lap[1:-1] - 2.0).max() < 1e-12
    # zero normal flux at the z faces: linear profile sees one face only
    lap = O.laplacian(G, z)
    assert np.abs(lap[0] - 1.0).max() < 1e-14 and np.abs(lap[-1] + 1.0).max() < 1e-14
    assert np.abs(lap[1:-1]).max() < 1e-14
    # periodic x Fourier mode: eigenvalue -4 sin^2(k/2)
    k = 2 * math.pi * 2 / 5
    f = np.cos(k * np.arange(5))[None, None, :] * np.ones((9, 4, 5))
    assert np.abs(O.laplacian(G, f) + 4 * math.sin(k / 2) ** 2 * f).max() < 1e-13


# --------------------------------------------------------- gradient flow (Eq. TDGL)

@pytest.mark.parametrize("volts", [False, True])
def test_energy_decreases(volts):
    G = mixed_grid(8, 6, 5, seed=3, eps=True, volts=volts)
    prm = O.Params(dt=0.01, rtol=1e-14)
    rng = np.random.default_rng(9)
    P = rng.uniform(-0.6, 0.6, (3,) + G.shape)
    phi = None
    F = [O.energy(G, prm, P)]
    for _ in range(12):
        P, phi, st, _ = O.step(G, prm, P, phi, 1)
        assert st == O.OK
        F.append(O.energy(G, prm, P))
    assert all(b < a for a, b in zip(F, F[1:]))


def test_driving_force_is_energy_gradient():
    """-dF/dP from central differences of the discrete energy equals the TDGL
    driving force recovered from one forward-Euler step."""
    G = mixed_grid(5, 4, 4, seed=21, eps=True, volts=True)
    prm = O.Params(a1=-1.0, a11=0.5, a12=0.8, g=0.5, dt=1.0, rtol=1e-14)
    rng = np.random.default_rng(4)
    P = rng.uniform(-0.5, 0.5, (3,) + G.shape)
    P1, _, _, _ = O.step(G, prm, P, None, 1)
    rate = P1 - P                       # dt L (-dF/dP) with dt = L = 1
    h = 1e-5
    for (c, z, y, x) in [(0, 0, 0, 0), (2, 3, 2, 1), (1, 1, 3, 4), (2, 0, 1, 2)]:
        Pp, Pm = P.copy(), P.copy()
        Pp[c, z, y, x] += h
        Pm[c, z, y, x] -= h
        dF = (O.energy(G, prm, Pp, 1e-14) - O.energy(G, prm, Pm, 1e-14)) / (2 * h)
        assert abs(dF + rate[c, z, y, x]) < 1e-7


# ----------------------------------------------------------------- symmetries

def test_periodic_shift_commutes_with_step():
    G = mixed_grid(8, 6, 5, seed=5, volts=True)
    prm = O.Params(rtol=1e-14)
    P = np.random.default_rng(1).uniform(-0.5, 0.5, (3,) + G.shape)
    P1, phi1, _, _ = O.step(G, prm, P, None, 3)
    sx, sy = 3, 2
    roll = lambda a, ax: np.roll(np.roll(a, sx, axis=ax[1]), sy, axis=ax[0])
    G2 = O.Grid(8, 6, 5, 1.0, False, roll(G.type_lo, (0, 1)), roll(G.volt_lo, (0, 1)),
                roll(G.type_hi, (0, 1)), roll(G.volt_hi, (0, 1)))
    P2, phi2, _, _ = O.step(G2, prm, roll(P, (2, 3)), None, 3)
    assert np.abs(P2 - roll(P1, (2, 3))).max() < 1e-12
    assert np.abs(phi2 - roll(phi1, (1, 2))).max() < 1e-12


def test_odd_symmetry():
    G = mixed_grid(6, 6, 4, seed=8, volts=True)
    Gm = O.Grid(6, 6, 4, 1.0, False, G.type_lo, -G.volt_lo, G.type_hi, -G.volt_hi)
    prm = O.Params(rtol=1e-14)
    P = np.random.default_rng(2).uniform(-0.5, 0.5, (3,) + G.shape)
    P1, phi1, _, _ = O.step(G, prm, P, None, 3)
    P2, phi2, _, _ = O.step(Gm, prm, -P, None, 3)
    assert np.abs(P1 + P2).max() < 1e-13
    assert np.abs(phi1 + phi2).max() < 1e-13


# ---------------------------------------------------------- solver edge cases

def test_noconv_returns_valid_state():
    G = mixed_grid(8, 8, 6, seed=1, volts=True)
    prm = O.Params(rtol=1e-14, maxit=1)
    P = np.random.default_rng(0).uniform(-0.5, 0.5, (3,) + G.shape)
    P1, phi, st, info = O.step(G, prm, P, None, 2)
    assert st == O.NOCONV and info["nonconverged"] == 2 and info["steps_done"] == 2
    assert np.isfinite(P1).all() and np.isfinite(phi).all()


def test_zero_rhs_gives_zero_potential():
    G = mixed_grid(4, 4, 4, seed=2)
    phi, st, it, rel = O.solve(G, np.zeros(G.shape), phi0=np.ones(G.shape))
    assert st == O.OK and it == 0 and np.abs(phi).max() == 0.0


def test_workload_generators_are_deterministic():
    a = W.film_fp64_grounded(8, 8, 8)
    b = W.film_fp64_grounded(8, 8, 8)
    assert np.array_equal(a.P0, b.P0)
    assert a.P0.min() >= -0.01 and a.P0.max() < 0.01
    # SplitMix64 published first output for seed 0 (state advanced once by the gamma)
    assert int(W.splitmix64(0, 0, 1)[0]) == 0xE220A8397B1DCDAF
    s = W.stripe_film(64, 64, 2, seed=2)
    assert np.allclose(np.linalg.norm(s - W.random_film(64, 64, 2, 2, -0.02, 0.02), axis=0), 1.0)
