"""Pins of the oracle's air layers (Section Results, open-circuit device: the
top layers are air with permittivity 1 against 100 in the film).  Air cells
carry no polarization; the film surface under the air is a free surface for
the gradient (wall) term.  Pins: the open-circuit Gauss law of a uniform film
(D = eps E + P = 0 everywhere, so E_z = -P_z/eps_film in the film and 0 in the
air), the Laplacian at the free surface, the gradient-flow structure (energy
decrease, force = -dF/dP by finite differences) and that air stays
unpolarized."""
import numpy as np
import pytest

import oracle as O


def air_grid(nx=6, ny=5, nz=10, n_air=4, eps_film=100.0, eps_air=1.0, top="open", seed=None):
    eps = np.full((nz, ny, nx), eps_film)
    eps[nz - n_air:] = eps_air
    tl = np.ones((ny, nx), np.int8)                   # grounded bottom electrode
    th = np.zeros((ny, nx), np.int8)                  # open top (Neumann)
    vl = np.zeros((ny, nx))
    vh = np.zeros((ny, nx))
    if seed is not None:
        rng = np.random.default_rng(seed)
        th = (rng.random((ny, nx)) < 0.5).astype(np.int8)
        vh = rng.uniform(-1, 1, (ny, nx))
    return O.Grid(nx, ny, nz, 1.0, False, tl, vl, th, vh, eps, n_air)


def test_open_circuit_gauss_law_with_air():
    G = air_grid()
    nz, na = G.nz, G.n_air
    P = np.zeros((3,) + G.shape)
    P[2, : nz - na] = 0.7
    phi, st, _, _ = O.solve_potential(G, P, rtol=1e-14)
    E = O.field(G, phi)
    assert st == O.OK
    film_inner = slice(1, nz - na - 1)
    assert np.abs(E[2, film_inner] + 0.7 / 100.0).max() < 1e-10
    assert np.abs(E[2, nz - na + 1:]).max() < 1e-10
    assert np.abs(E[0]).max() < 1e-12 and np.abs(E[1]).max() < 1e-12


def test_laplacian_has_a_free_surface_under_the_air():
    G = air_grid(n_air=3)
    f = np.zeros(G.shape)
    for z in range(G.nz):
        f[z] = float(z)
    lap = O.laplacian(G, f)
    top = G.nz - G.n_air - 1
    assert np.abs(lap[1:top]).max() < 1e-14              # linear in the film interior
    assert np.abs(lap[top] + 1.0).max() < 1e-14          # only the face below: (top-1) - top
    assert np.abs(lap[0] - 1.0).max() < 1e-14            # bottom: zero flux through the grid face
    assert np.abs(lap[top + 1:]).max() == 0.0            # air


def test_air_stays_unpolarized_and_the_film_evolves():
    G = air_grid(seed=3)
    prm = O.Params(dt=0.01, rtol=1e-13)
    P0 = np.random.default_rng(1).uniform(-0.5, 0.5, (3,) + G.shape)
    P0[:, G.nz - G.n_air:] = 0.0
    for scheme in ("euler", "heun"):
        P, _, st, _ = O.step_ex(G, prm, P0, None, 4, scheme, sigma=0.1, seed=2)
        assert st == O.OK
        assert np.abs(P[:, G.nz - G.n_air:]).max() == 0.0
        assert np.abs(P[:, : G.nz - G.n_air] - P0[:, : G.nz - G.n_air]).max() > 1e-3


def test_energy_decreases_with_air():
    G = air_grid()
    prm = O.Params(dt=0.01, rtol=1e-14)
    P = np.random.default_rng(5).uniform(-0.6, 0.6, (3,) + G.shape)
    P[:, G.nz - G.n_air:] = 0.0
    phi = None
    F = [O.energy(G, prm, P)]
    for _ in range(10):
        P, phi, st, _ = O.step(G, prm, P, phi, 1)
        F.append(O.energy(G, prm, P))
    assert all(b < a for a, b in zip(F, F[1:]))


def test_driving_force_is_the_energy_gradient_with_air():
    G = air_grid(nx=4, ny=4, nz=7, n_air=3, seed=7)
    prm = O.Params(dt=1.0, rtol=1e-14)
    P = np.random.default_rng(4).uniform(-0.5, 0.5, (3,) + G.shape)
    P[:, G.nz - G.n_air:] = 0.0
    P1, _, _, _ = O.step(G, prm, P, None, 1)
    rate = P1 - P
    h = 1e-5
    top = G.nz - G.n_air - 1
    for (c, z, y, x) in [(2, top, 1, 2), (0, top, 3, 0), (1, 0, 2, 2), (2, top - 1, 0, 3)]:
        Pp, Pm = P.copy(), P.copy()
        Pp[c, z, y, x] += h
        Pm[c, z, y, x] -= h
        dF = (O.energy(G, prm, Pp, 1e-14) - O.energy(G, prm, Pm, 1e-14)) / (2 * h)
        assert abs(dF + rate[c, z, y, x]) < 1e-7
