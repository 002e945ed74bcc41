"""GPU parity of the thermal random force (Eq. TDGL's zeta: Philox4x32-10 +
Box-Muller per cell, component and step) against the oracle's stream.  FP64
bar 1e-10 on P and phi, FP32 1e-4 on P."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1202_6116_gb300 import build as B
from paper_1202_6116_gb300 import pf
from paper_1202_6116_gb300 import workloads as W
from paper_1202_6116_gb300.batch import Batch
from paper_1202_6116_gb300.film import Film

from helpers import mixed_workload, oracle_grid, oracle_params, relerr

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pf.lib()


def gpu_noisy(w, chunks, sigma, seed, **over):
    f = Film(w, **over)
    f.set_noise(sigma, seed)
    infos = [f.step(c)[1] for c in chunks]
    P, phi = f.numpy()
    f.close()
    return P, phi, infos


@pytest.mark.parametrize("scheme,every,solver", [("euler", 1, "pcg"), ("heun", 2, "pcg"), ("euler", 1, "mg")])
def test_fp64_noise_matches_oracle(scheme, every, solver):
    nx, ny, nz = (40, 24, 12) if solver == "mg" else (37, 22, 11)
    w = mixed_workload(nx, ny, nz, 51, steps=7, rtol=1e-13).with_(solver=solver, maxit=3000)
    integ = pf.PF_HEUN if scheme == "heun" else pf.PF_EULER
    P, phi, _ = gpu_noisy(w, [3, 4], 0.3, 1234567890123, integrator=integ, poisson_every=every)
    Po, phio, st, _ = O.step_ex(oracle_grid(w), oracle_params(w, 1e-14), w.P0, None, 7, scheme, every,
                                sigma=0.3, seed=1234567890123)
    assert st == O.OK
    assert relerr(P, Po) <= FP64_TOL
    assert relerr(phi, phio) <= FP64_TOL
    Pq, _, _, _ = O.step_ex(oracle_grid(w), oracle_params(w, 1e-14), w.P0, None, 7, scheme, every)
    assert np.abs(Po - Pq).max() > 1e-3                  # the noise is really there


def test_fp32_noise_vs_fp64_oracle():
    w = W.film_strip_fp32(64, 64, 16, steps=20)
    P, _, _ = gpu_noisy(w, [20], 0.2, 99)
    Po, _, st, _ = O.step_ex(oracle_grid(w), oracle_params(w, 1e-12), w.P0, None, 20, sigma=0.2, seed=99)
    assert st == O.OK
    assert relerr(P, Po) <= FP32_TOL


def test_noise_graph_host_and_tiling_agree():
    """Graph-launched, host-driven and re-tiled runs draw the same stream."""
    w = mixed_workload(48, 32, 8, 53, steps=5, rtol=1e-13)
    a, _, ia = gpu_noisy(w, [5], 0.25, 7)
    f = Film(w)
    f.set_noise(0.25, 7)
    pf.pf_profile_enable(f.ctx, 1)
    _, ib = f.step(5)
    b = f.numpy()[0]
    f.close()
    c, _, _ = gpu_noisy(w, [5], 0.25, 7)
    assert ia[0]["graph_steps"] == 5 and ib["graph_steps"] == 0
    assert np.array_equal(a, b) and np.array_equal(a, c)
    f = Film(w)
    f.set_noise(0.25, 7)
    pf.pf_set_tiling(f.ctx, 1, 3, 0)
    f.step(5)
    d = f.numpy()[0]
    f.close()
    assert relerr(d, a) <= 1e-12


def test_noise_in_a_batch_equals_films_alone():
    ws = W.film_batch_hysteresis(nfilms=2, seed=31, steps=6, shapes=((32, 32, 16), (16, 16, 8)), precision="fp64",
                                 rtol=1e-12)
    films = [Film(w) for w in ws]
    for i, f in enumerate(films):
        f.set_noise(0.1 * (i + 1), 40 + i)
    b = Batch(films, max_records=6)
    b.step(6)
    got = [f.numpy()[0] for f in films]
    b.close()
    for f in films:
        f.close()
    for i, w in enumerate(ws):
        f = Film(w)
        f.set_noise(0.1 * (i + 1), 40 + i)
        f.step(6)
        assert np.array_equal(f.numpy()[0], got[i])
        f.close()


def test_noise_arguments_and_adjoint():
    w = mixed_workload(16, 16, 8, 5, steps=1)
    f = Film(w, flags=pf.PF_FLAG_ADJOINT)
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(pf.PfError):
            f.set_noise(bad, 1)
    f.set_noise(0.1, 1)
    lam = torch.zeros_like(f.P)
    with pytest.raises(pf.PfError) as e:
        pf.pf_adjoint_step(f.ctx, lam, torch.zeros_like(f.P), torch.zeros(4, dtype=torch.float64, device=f.P.device))
    assert e.value.status == pf.PF_ERR_NOTIMPL
    f.set_noise(0.0, 1)                                 # off again: the adjoint is available
    pf.pf_adjoint_step(f.ctx, lam, torch.zeros_like(f.P), torch.zeros(4, dtype=torch.float64, device=f.P.device))
    f.close()
