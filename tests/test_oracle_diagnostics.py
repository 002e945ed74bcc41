"""Pins of the oracle's run diagnostics (mean P, switched-domain fraction and
the three energy terms of Eqs. F_bulk, F_grad and F_elec) against closed
forms and the generator's own stripe choices."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1202_6116_gb300 import workloads as W


def test_uniform_r_state_closed_forms():
    """Uniform R-phase film between grounded electrodes: no field, no gradient
    energy, Landau energy N f(P_R) with f(P_R) = -0.576923 (a12 < 2 a11)."""
    nx, ny, nz = 6, 5, 4
    G = O.Grid(nx, ny, nz, type_lo=np.ones((ny, nx)), type_hi=np.ones((ny, nx)))
    prm = O.Params()
    p = math.sqrt(1.0 / (2.0 * (0.5 + 0.8)))
    P = np.empty((3,) + G.shape)
    P[0], P[1], P[2] = p, -p, p
    phi, st, _, _ = O.solve_potential(G, P)
    d = O.diagnostics(G, prm, P, phi)
    n = nx * ny * nz
    assert abs(d["mean_px"] - p) < 1e-15 and abs(d["mean_py"] + p) < 1e-15 and abs(d["mean_pz"] - p) < 1e-15
    assert d["switched_fraction"] == 1.0
    assert abs(d["f_landau"] - n * (-3.0 / (4.0 * (0.5 + 0.8)))) < 1e-12
    assert d["f_grad"] == 0.0 and abs(d["f_elec"]) < 1e-15


@pytest.mark.parametrize("dx", [1.0, 0.5])
def test_gradient_energy_of_a_sine_mode(dx):
    """P_y = A sin(2 pi m x / nx): sum_x (P(x+1) - P(x))^2 = 2 nx A^2 sin^2(pi m / nx)
    per (y, z) line; the z-faces add nothing (no z variation)."""
    nx, ny, nz, m, A = 12, 3, 4, 2, 0.3
    G = O.Grid(nx, ny, nz, dx=dx)
    prm = O.Params(g=0.7)
    P = np.zeros((3,) + G.shape)
    P[1] = A * np.sin(2 * math.pi * m * np.arange(nx) / nx)[None, None, :]
    d = O.diagnostics(G, prm, P, np.zeros(G.shape))
    want = 0.5 * 0.7 * ny * nz * 2 * nx * A * A * math.sin(math.pi * m / nx) ** 2 / dx ** 2
    assert abs(d["f_grad"] - want) < 1e-12 * want


def test_switched_fraction_counts_stripes():
    """Stripe film: P_x > 0.3 exactly in the stripes whose <111> variant has +x
    (the noise of 0.02 cannot flip a component of size 0.577)."""
    nx, ny, nz, width = 64, 48, 3, 16
    P = W.stripe_film(nx, ny, nz, seed=5, width=width)
    sid = (np.arange(nx)[None, :] + np.arange(ny)[:, None]) // width
    pick = np.minimum((W.uniform(5 + 1000, int(sid.max()) + 1) * 4).astype(np.int64), 3)
    plus_x = np.array([1, 0, 0, 1])[pick[sid]]              # variants (+-1, +-1, -1): x sign per index
    G = O.Grid(nx, ny, nz)
    d = O.diagnostics(G, O.Params(), P, np.zeros(G.shape))
    assert d["switched_fraction"] == plus_x.mean()


@pytest.mark.parametrize("eps", [False, True])
def test_terms_add_up_to_the_free_energy(eps):
    """Electrodes at 0 V, phi the potential of P: f_landau + f_grad + f_elec is
    the free energy whose gradient is the TDGL driving force."""
    rng = np.random.default_rng(8)
    ny, nx, nz = 5, 7, 4
    tl = (rng.random((ny, nx)) < 0.5).astype(np.int8)
    th = (rng.random((ny, nx)) < 0.5).astype(np.int8)
    e = rng.uniform(0.5, 3.0, (nz, ny, nx)) if eps else None
    G = O.Grid(nx, ny, nz, type_lo=tl, type_hi=th, eps=e)
    prm = O.Params()
    P = rng.uniform(-0.6, 0.6, (3,) + G.shape)
    phi, st, _, _ = O.solve_potential(G, P)
    d = O.diagnostics(G, prm, P, phi)
    F = O.energy(G, prm, P)
    assert abs(d["f_landau"] + d["f_grad"] + d["f_elec"] - F) < 1e-12 * abs(F)
    assert d["f_elec"] > 0.0      # -1/2 P.E >= 0: the depolarizing field opposes P
