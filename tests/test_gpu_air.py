"""GPU parity of the air layers (the paper's open-circuit device: air with
permittivity 1 over a film with 100, P = 0 in the air, a free film surface
for the wall term) against the FP64 oracle.  FP64 bar 1e-10 on P and phi,
FP32 1e-4 on P."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1202_6116_gb300 import build as B
from paper_1202_6116_gb300 import pf
from paper_1202_6116_gb300 import workloads as W
from paper_1202_6116_gb300.film import Film

from helpers import oracle_grid, oracle_params, relerr

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pf.lib()


@pytest.mark.parametrize("shape,n_air,scheme,sigma", [((32, 24, 13), 4, "euler", 0.0),
                                                      ((36, 20, 11), 3, "heun", 0.2)])
def test_fp64_open_air_matches_oracle(shape, n_air, scheme, sigma):
    nx, ny, nz = shape
    w = W.film_open_air(nx, ny, nz, n_air=n_air, steps=8, precision="fp64").with_(rtol=1e-13)
    f = Film(w, integrator=pf.PF_HEUN if scheme == "heun" else pf.PF_EULER)
    if sigma:
        f.set_noise(sigma, 77)
    f.step(3)
    f.step(5)
    P, phi = f.numpy()
    d = f.diagnostics(0.3)
    f.close()
    Po, phio, st, _ = O.step_ex(oracle_grid(w), oracle_params(w, 1e-14), w.P0, None, 8, scheme, sigma=sigma, seed=77)
    assert st == O.OK
    assert np.abs(P[:, nz - n_air:]).max() == 0.0
    assert relerr(P, Po) <= FP64_TOL
    assert relerr(phi, phio) <= FP64_TOL
    o = O.diagnostics(oracle_grid(w), oracle_params(w), P, phi, 0.3)
    for k in ("f_landau", "f_grad", "f_elec"):
        assert abs(d[k] - o[k]) <= FP64_TOL * max(abs(o[k]), 1e-30), (k, d[k], o[k])


def test_fp32_open_air_vs_fp64_oracle():
    w = W.film_open_air(64, 64, 21, n_air=5, steps=30)
    f = Film(w)
    f.step(30)
    P, _ = f.numpy()
    f.close()
    Po, _, st, _ = O.step_ex(oracle_grid(w), oracle_params(w, 1e-12), w.P0, None, 30)
    assert st == O.OK
    assert np.abs(P[:, w.nz - w.n_air:]).max() == 0.0
    assert relerr(P, Po) <= FP32_TOL


def test_air_layers_and_the_adjoint():
    w = W.film_open_air(16, 16, 9, n_air=3, steps=1, precision="fp64")
    f = Film(w, flags=pf.PF_FLAG_ADJOINT)
    lam = torch.zeros_like(f.P)
    with pytest.raises(pf.PfError) as e:
        pf.pf_adjoint_step(f.ctx, lam, torch.zeros_like(f.P), torch.zeros(4, dtype=torch.float64, device=f.P.device))
    assert e.value.status == pf.PF_ERR_NOTIMPL
    f.close()


@pytest.mark.parametrize("shape,n_air", [((32, 24, 13), 4), ((32, 32, 16), 5)])
def test_mg_open_air_matches_oracle(shape, n_air):
    """The permittivity-aware multigrid preconditioner (coarse eps = mean of
    the children, harmonic-mean faces on every level) on the open-air film:
    FP64 parity with the oracle's Jacobi-PCG at tight tolerances."""
    nx, ny, nz = shape
    w = W.film_open_air(nx, ny, nz, n_air=n_air, steps=6, precision="fp64").with_(rtol=1e-13, solver="mg",
                                                                                    maxit=400)
    f = Film(w)
    st, info = f.step(6)
    P, phi = f.numpy()
    f.close()
    Po, phio, sto, _ = O.step_ex(oracle_grid(w), oracle_params(w, 1e-14), w.P0, None, 6)
    assert st == pf.PF_OK and sto == O.OK
    assert relerr(P, Po) <= FP64_TOL
    assert relerr(phi, phio) <= FP64_TOL


def test_mg_random_permittivity_matches_oracle():
    from helpers import mixed_workload
    w = mixed_workload(32, 16, 8, 43, eps=True, steps=4, rtol=1e-13).with_(solver="mg", maxit=400)
    f = Film(w)
    st, _ = f.step(4)
    P, phi = f.numpy()
    f.close()
    Po, phio, sto, _ = O.step(oracle_grid(w), oracle_params(w, 1e-14), w.P0, None, 4)
    assert st == pf.PF_OK
    assert relerr(P, Po) <= FP64_TOL
    assert relerr(phi, phio) <= FP64_TOL


def test_mg_cuts_the_air_film_iterations():
    """At the open-air recipe's 100:1 permittivity contrast, multigrid needs
    a small fraction of Jacobi-PCG's iterations per solve, and the FP32
    results agree with the FP64 oracle."""
    w = W.film_open_air(64, 64, 37, n_air=5, steps=10)
    its = {}
    Ps = {}
    for solver, maxit in (("pcg", 5000), ("mg", 400)):
        f = Film(w.with_(solver=solver, maxit=maxit))
        st, info = f.step(10)
        assert st == pf.PF_OK
        its[solver] = info["total_iters"] / info["solves"]
        Ps[solver], _ = f.numpy()
        f.close()
    print("iterations per solve: Jacobi %.1f, multigrid %.1f" % (its["pcg"], its["mg"]))
    assert its["mg"] <= 30
    assert its["mg"] <= 0.25 * its["pcg"]
    Po, _, st, _ = O.step_ex(oracle_grid(w), oracle_params(w, 1e-12), w.P0, None, 10)
    assert relerr(Ps["mg"], Po) <= FP32_TOL
