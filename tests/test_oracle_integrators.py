"""Pins of the oracle's time-integration options (Section Time Integration:
forward Euler and the predictor-corrector the paper calls velocity Verlet;
Section Numerical Performance: long-range terms solved every few steps).

The pins are independent of the oracle's own stepping code: a scalar ODE
whose exact solution is known (second-order convergence of the corrector),
the scalar recurrence of the predictor-corrector written out here, and
compositions of the oracle's separately pinned operators (potential solve,
field, Landau force, Laplacian) in the step order the paper states.
"""
import math

import numpy as np
import pytest

import oracle as O


def uniform_field(G, vec):
    P = np.zeros((3,) + G.shape)
    for c in range(3):
        P[c] = vec[c]
    return P


def strip_grid(nx, ny, nz, v=1.5):
    tl = np.zeros((ny, nx), np.int8)
    th = np.zeros((ny, nx), np.int8)
    vh = np.zeros((ny, nx))
    th[:, : nx // 4] = 1
    vh[:, : nx // 4] = v
    th[:, nx // 2: 3 * nx // 4] = 1
    vh[:, nx // 2: 3 * nx // 4] = -v
    tl[:, :] = 1
    return O.Grid(nx, ny, nz, 1.0, False, tl, None, th, vh)


def rate_from_operators(G, prm, P, phi):
    """L(-df/dP + g Lap P + E(phi)) from the pinned operators (Eq. TDGL)."""
    h = O.landau_force(P, prm)
    lap = np.stack([O.laplacian(G, P[c]) for c in range(3)])
    E = O.field(G, phi)
    return prm.L * (-h + prm.g * lap + E)


def test_euler_every_step_is_the_plain_step():
    G = strip_grid(8, 6, 5)
    prm = O.Params(dt=0.01, rtol=1e-13)
    P0 = np.random.default_rng(1).uniform(-0.4, 0.4, (3,) + G.shape)
    a = O.step(G, prm, P0, None, 4)
    b = O.step_ex(G, prm, P0, None, 4, "euler", 1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[3]["total_iters"] == b[3]["total_iters"]


def test_rate_matches_operator_composition():
    G = strip_grid(8, 6, 5)
    prm = O.Params(dt=0.01, L=1.7, g=0.3, rtol=1e-13)
    rng = np.random.default_rng(2)
    P = rng.uniform(-0.5, 0.5, (3,) + G.shape)
    phi = rng.uniform(-1, 1, G.shape)
    assert np.abs(O.rate(G, prm, P, phi) - rate_from_operators(G, prm, P, phi)).max() < 1e-14


@pytest.mark.parametrize("direction,coef", [((1, 1, 1), 5.2), ((0, 0, 1), 2.0)])
def test_heun_homogeneous_recurrence(direction, coef):
    """Uniform P between grounded electrodes has phi = 0, so every nonzero
    component follows the scalar predictor-corrector recurrence of
    p' = 2 p - coef p^3 (coef = 4 a11 + 2 a12 (#nonzero - 1), Eq. F_bulk)."""
    G = O.Grid(6, 5, 4, type_lo=np.ones((5, 6)), type_hi=np.ones((5, 6)))
    dt, p = 0.02, 0.1
    prm = O.Params(dt=dt, rtol=1e-14)
    P, phi, st, info = O.step_ex(G, prm, uniform_field(G, [p * d for d in direction]), None, 40, "heun")
    f = lambda q: 2 * q - coef * q ** 3
    for _ in range(40):
        pp = p + dt * f(p)
        p = p + dt * 0.5 * (f(p) + f(pp))
    for c in range(3):
        assert np.abs(P[c] - p * direction[c]).max() < 1e-15
    assert info["total_iters"] == 0 and st == O.OK


def test_heun_second_order_on_the_logistic_law():
    """u = p^2 obeys u' = 4u (1 - u/u_inf) (u_inf = 1/2.6) for a uniform [111]
    film: halving dt quarters the predictor-corrector's error (forward Euler:
    halves it)."""
    G = O.Grid(2, 2, 2, periodic_z=True)
    uinf, u0, T = 1.0 / 2.6, 0.01, 2.0
    exact = uinf / (1 + (uinf / u0 - 1) * math.exp(-4 * T))
    errs = {"heun": [], "euler": []}
    for scheme in errs:
        for dt in (0.04, 0.02, 0.01):
            P, _, _, _ = O.step_ex(G, O.Params(dt=dt), uniform_field(G, [math.sqrt(u0)] * 3), None,
                                   int(round(T / dt)), scheme)
            errs[scheme].append(abs(P[0, 0, 0, 0] ** 2 - exact))
    h = errs["heun"]
    assert h[0] / h[1] == pytest.approx(4.0, rel=0.1) and h[1] / h[2] == pytest.approx(4.0, rel=0.1)
    e = errs["euler"]
    assert e[1] / e[2] == pytest.approx(2.0, rel=0.1)
    assert h[2] < e[2] / 20


def test_heun_with_field_matches_operator_composition():
    """Two predictor-corrector steps with strip electrodes: each stage solves
    the potential of its own state (warm-started from the last one)."""
    G = strip_grid(10, 6, 5)
    prm = O.Params(dt=0.02, rtol=1e-13)
    P0 = np.random.default_rng(3).uniform(-0.5, 0.5, (3,) + G.shape)
    P, phi, st, info = O.step_ex(G, prm, P0, None, 2, "heun")
    Pc, ph = P0.copy(), np.zeros(G.shape)
    for _ in range(2):
        ph, s1, _, _ = O.solve_potential(G, Pc, ph, rtol=prm.rtol)
        Rc = rate_from_operators(G, prm, Pc, ph)
        Pp = Pc + prm.dt * Rc
        ph, s2, _, _ = O.solve_potential(G, Pp, ph, rtol=prm.rtol)
        Rp = rate_from_operators(G, prm, Pp, ph)
        Pc = Pc + prm.dt * (0.5 * (Rc + Rp))
    assert st == O.OK
    assert np.abs(P - Pc).max() < 1e-13 * np.abs(Pc).max()
    assert np.abs(phi - ph).max() < 1e-13 * np.abs(ph).max()


@pytest.mark.parametrize("scheme,every,n0", [("euler", 3, 0), ("euler", 5, 3), ("heun", 2, 1)])
def test_long_range_every_k_steps_holds_the_field(scheme, every, n0):
    """The potential is solved only on global steps that are multiples of
    every; in between, the update (both stages for the predictor-corrector)
    uses the last potential solved."""
    G = strip_grid(8, 6, 5)
    prm = O.Params(dt=0.02, rtol=1e-13)
    rng = np.random.default_rng(4)
    P0 = rng.uniform(-0.5, 0.5, (3,) + G.shape)
    phi0 = rng.uniform(-0.2, 0.2, G.shape)
    nsteps = 6
    P, phi, st, info = O.step_ex(G, prm, P0, phi0, nsteps, scheme, every, n0)
    Pc, ph, solves = P0.copy(), phi0.copy(), 0
    for s in range(nsteps):
        refresh = (n0 + s) % every == 0
        if refresh:
            ph, _, _, _ = O.solve_potential(G, Pc, ph, rtol=prm.rtol)
            solves += 1
        Rc = rate_from_operators(G, prm, Pc, ph)
        if scheme == "heun":
            Pp = Pc + prm.dt * Rc
            if refresh:
                ph, _, _, _ = O.solve_potential(G, Pp, ph, rtol=prm.rtol)
                solves += 1
            Pc = Pc + prm.dt * (0.5 * (Rc + rate_from_operators(G, prm, Pp, ph)))
        else:
            Pc = Pc + prm.dt * Rc
    assert st == O.OK
    assert np.abs(P - Pc).max() < 1e-13 * np.abs(Pc).max()
    assert np.abs(phi - ph).max() < 1e-13 * np.abs(ph).max()
    assert solves > 0 and info["total_iters"] > 0


def test_heun_energy_decreases():
    """The predictor-corrector is a consistent gradient-flow integrator: at a
    small step the free energy decreases with grounded electrodes."""
    G = O.Grid(8, 6, 5, type_lo=np.ones((6, 8)), type_hi=np.ones((6, 8)))
    prm = O.Params(dt=0.02, rtol=1e-14)
    P = np.random.default_rng(5).uniform(-0.6, 0.6, (3,) + G.shape)
    phi = None
    F = [O.energy(G, prm, P)]
    for _ in range(10):
        P, phi, st, _ = O.step_ex(G, prm, P, phi, 1, "heun")
        F.append(O.energy(G, prm, P))
    assert all(b < a for a, b in zip(F, F[1:]))


@pytest.mark.parametrize("kind", ["mixed", "air", "periodic"])
def test_rate_at_samples_equals_the_whole_grid_rate(kind):
    """or_rate_at (used to check large GPU states at sampled cells) evaluates
    the same per-cell terms as or_rate."""
    rng = np.random.default_rng(8)
    if kind == "air":
        eps = rng.uniform(1.0, 3.0, (7, 6, 9))
        G = O.Grid(9, 6, 7, 1.0, False, np.ones((6, 9), np.int8), None, np.zeros((6, 9), np.int8), None, eps, 2)
    elif kind == "periodic":
        G = O.Grid(9, 6, 7, 1.0, True)
    else:
        G = strip_grid(9, 6, 7)
    prm = O.Params(g=0.3, L=1.3)
    P = rng.uniform(-0.5, 0.5, (3,) + G.shape)
    if kind == "air":
        P[:, G.nz - G.n_air:] = 0.0
    phi = rng.uniform(-1, 1, G.shape)
    R = O.rate(G, prm, P, phi).reshape(3, -1)
    cells = np.arange(G.n)
    assert np.array_equal(O.rate_at(G, prm, P, phi, cells), R.T)
