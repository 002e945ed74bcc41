"""Pins of the oracle's thermal random force (Eq. TDGL: zeta with zero mean
and Gaussian variance), drawn per cell, component and step from a
counter-based generator (Philox4x32-10 with the Box-Muller transform).

The pins are independent of the generator's code: the generator's published
known-answer values (tests/golden/philox4x32_10_kat.json); the draws are
standard normal and uncorrelated; one step of the free process
has variance sigma^2 dt; a linear restoring force gives the Ornstein-Uhlenbeck
process, whose discrete stationary variance has a closed form; the
predictor-corrector adds the same increment in both stages.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

scipy_stats = pytest.importorskip("scipy.stats")


def test_philox_known_answers():
    """Philox4x32-10 as published (Salmon et al., SC11): the known-answer
    outputs for zero, all-ones and pi-digit counters and keys.  A wrong
    multiplier, Weyl constant, round count or word order fails them."""
    kat = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")))
    for v in kat["vectors"]:
        c = [int(w, 16) for w in v["counter"]]
        k = [int(w, 16) for w in v["key"]]
        cell, step, seed = c[0] | c[1] << 32, c[2] | c[3] << 32, k[0] | k[1] << 32
        assert O.philox(seed, step, cell) == [int(w, 16) for w in v["out"]]


def test_draws_are_standard_normal_and_uncorrelated():
    cells = np.arange(6000)
    a = np.array([O.gauss4(11, 0, c) for c in cells])           # (cells, 4)
    b = np.array([O.gauss4(11, 1, c) for c in cells])           # next step
    x = a.ravel()
    n = x.size
    assert abs(x.mean()) < 4 / math.sqrt(n)
    assert abs(x.var() - 1.0) < 4 * math.sqrt(2.0 / n)
    assert scipy_stats.kstest(x, "norm").pvalue > 1e-3
    lim = 4 / math.sqrt(len(cells))
    for i in range(4):
        for j in range(i):
            assert abs(np.corrcoef(a[:, i], a[:, j])[0, 1]) < lim        # components
        assert abs(np.corrcoef(a[:-1, i], a[1:, i])[0, 1]) < lim        # neighbouring cells
        assert abs(np.corrcoef(a[:, i], b[:, i])[0, 1]) < lim           # consecutive steps
    c = np.array([O.gauss4(12, 0, k) for k in cells])                 # another seed
    assert abs(np.corrcoef(a[:, 0], c[:, 0])[0, 1]) < lim
    assert np.array_equal(np.array([O.gauss4(11, 0, k) for k in cells[:50]]), a[:50])


def free_film(n=16):
    """No deterministic force: Landau and gradient coefficients 0, and a huge
    permittivity, so that the field of any P is negligible (~1e-12)."""
    G = O.Grid(n, n, n, type_lo=np.ones((n, n)), type_hi=np.ones((n, n)), eps=np.full((n, n, n), 1e12))
    return G


def test_one_step_of_the_free_process_has_variance_sigma2_dt():
    G = free_film()
    sigma, dt = 0.3, 0.04
    prm = O.Params(a1=0.0, a11=0.0, a12=0.0, g=0.0, dt=dt, rtol=1e-12)
    P, _, st, _ = O.step_ex(G, prm, np.zeros((3,) + G.shape), None, 1, sigma=sigma, seed=5)
    x = P.ravel()
    assert st == O.OK
    assert abs(x.mean()) < 4 * sigma * math.sqrt(dt / x.size)
    assert x.var() / (sigma ** 2 * dt) == pytest.approx(1.0, abs=4 * math.sqrt(2.0 / x.size))


def test_ornstein_uhlenbeck_stationary_variance():
    """f = a1 sum P_i^2 only: each component follows p <- (1 - 2 a1 L dt) p +
    sigma sqrt(dt) g, whose stationary variance is sigma^2 dt / (1 - (1 - 2 a1 L dt)^2)."""
    G = free_film()
    sigma, dt, a1, L = 0.5, 0.05, 0.5, 1.0
    prm = O.Params(a1=a1, a11=0.0, a12=0.0, g=0.0, L=L, dt=dt, rtol=1e-12)
    P, _, st, _ = O.step_ex(G, prm, np.zeros((3,) + G.shape), None, 300, sigma=sigma, seed=21)
    rho = 1.0 - 2.0 * a1 * L * dt
    v = sigma ** 2 * dt / (1.0 - rho ** 2)
    x = P.ravel()
    assert st == O.OK
    assert x.var() / v == pytest.approx(1.0, abs=0.06)
    assert abs(x.mean()) < 4 * math.sqrt(v / x.size)


def test_predictor_corrector_adds_the_same_increment():
    """With no deterministic force the corrected state is P + sigma sqrt(dt) g,
    as in forward Euler: both stages see one draw."""
    G = free_film(8)
    prm = O.Params(a1=0.0, a11=0.0, a12=0.0, g=0.0, dt=0.02, rtol=1e-12)
    P0 = np.random.default_rng(2).uniform(-0.1, 0.1, (3,) + G.shape)
    e, _, _, _ = O.step_ex(G, prm, P0, None, 3, "euler", sigma=0.4, seed=9)
    h, _, _, _ = O.step_ex(G, prm, P0, None, 3, "heun", sigma=0.4, seed=9)
    assert np.abs(e - h).max() < 1e-10
    assert np.abs(e - P0).max() > 0.01


def test_noise_stream_follows_the_global_step():
    """Splitting a run (n0 offsets) reproduces the single run; another seed differs."""
    G = O.Grid(8, 6, 5, type_lo=np.ones((6, 8)), type_hi=np.ones((6, 8)))
    prm = O.Params(dt=0.01, rtol=1e-13)
    P0 = np.random.default_rng(3).uniform(-0.3, 0.3, (3,) + G.shape)
    a, pa, _, _ = O.step_ex(G, prm, P0, None, 6, sigma=0.2, seed=4)
    b1, pb, _, _ = O.step_ex(G, prm, P0, None, 2, sigma=0.2, seed=4)
    b, pb, _, _ = O.step_ex(G, prm, b1, pb, 4, n0=2, sigma=0.2, seed=4)
    assert np.abs(a - b).max() < 1e-12
    c, _, _, _ = O.step_ex(G, prm, P0, None, 6, sigma=0.2, seed=5)
    assert np.abs(a - c).max() > 1e-3
    d, _, _, _ = O.step_ex(G, prm, P0, None, 6, sigma=0.0, seed=4)
    e, _, _, _ = O.step_ex(G, prm, P0, None, 6)
    assert np.array_equal(d, e)
