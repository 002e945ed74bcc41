"""Parity at the benchmark's full size (the 1024 x 1024 x 128 tip-electrode
film, multigrid-preconditioned CG, default tiling, graph-launched steps): the
oracle cannot run the whole film, so it checks what it can compute one by one
or what holds at any size.
  - The TDGL update at sampled cells (faces, electrode edges, interior):
    P_{n+1} = P_n + dt R(P_n, phi_n), R from the oracle's per-cell rate.
  - The Poisson solve's true FP64 relative residual ||b - A phi|| / ||b|| from
    the oracle's right-hand side and operator over the whole grid.
  - FP32 against FP64 after the same steps."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1202_6116_gb300 import build as B
from paper_1202_6116_gb300 import pf
from paper_1202_6116_gb300 import workloads as W
from paper_1202_6116_gb300.film import Film

from helpers import oracle_grid, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pf.lib()


@pytest.fixture(scope="module")
def tip():
    return W.film_tip_fp32()


def sample_cells(w, m=3000, seed=0):
    rng = np.random.default_rng(seed)
    nx, ny, nz = w.nx, w.ny, w.nz
    zs = np.concatenate([[0, 1, nz - 2, nz - 1] * (m // 8), rng.integers(0, nz, m - 4 * (m // 8))])
    ys = rng.integers(0, ny, len(zs))
    xs = rng.integers(0, nx, len(zs))
    # the tip electrode's edge rows and the tile seams
    s = nx // 8
    x0 = (nx - s) // 2
    xs[: m // 10] = np.where(rng.random(m // 10) < 0.5, x0, x0 + s - 1)
    xs[m // 10: m // 5] = rng.choice([0, 63, 64, nx - 1], m // 10)
    return (zs.astype(np.int64) * ny + ys) * nx + xs


def run_two_steps(w, precision):
    f = Film(w.with_(precision=precision))
    f.step(1)
    P1 = f.P.double().cpu().numpy()
    _, info = f.step(1)
    P2 = f.P.double().cpu().numpy()
    phi1 = f.phi.double().cpu().numpy()                 # the potential of P1
    st, sinfo = f.solve_potential()
    phi2 = f.phi.double().cpu().numpy()                 # the potential of P2
    f.close()
    assert info["graph_steps"] == 1 and info["status"] == pf.PF_OK
    return P1, P2, phi1, phi2, sinfo


@pytest.fixture(scope="module")
def runs(tip):
    return {prec: run_two_steps(tip, prec) for prec in ("fp64", "fp32")}


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_full_size_tdgl_update_at_sampled_cells(tip, runs, precision, tol):
    P1, P2, phi1, _, _ = runs[precision]
    G = oracle_grid(tip)
    cells = sample_cells(tip)
    R = O.rate_at(G, oracle_params(tip), P1, phi1, cells)
    n = tip.n
    got = P2.reshape(3, n)[:, cells].T
    want = P1.reshape(3, n)[:, cells].T + tip.dt * R
    assert np.abs(got - want).max() <= tol * np.abs(P1).max()


def test_full_size_poisson_residual_fp64(tip, runs):
    _, P2, _, phi2, info = runs["fp64"]
    G = oracle_grid(tip)
    b = O.rhs(G, P2)
    r = b - O.apply(G, phi2)
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert info["last_relres"] < tip.rtol
    assert rel <= 1.01 * tip.rtol


def test_full_size_fp32_against_fp64(runs):
    P64 = runs["fp64"][1]
    P32 = runs["fp32"][1]
    assert np.abs(P32 - P64).max() <= 1e-4 * np.abs(P64).max()
