"""GPU parity of the time-integration options against the FP64 oracle
(Section Time Integration: the predictor-corrector scheme; Section Numerical
Performance: the long-range potential solved every k steps).  Same error
metric and bars as the forward-Euler parity tests: FP64 1e-10 on P and phi,
FP32 1e-4 on P."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1202_6116_gb300 import build as B
from paper_1202_6116_gb300 import pf
from paper_1202_6116_gb300 import workloads as W
from paper_1202_6116_gb300.film import Film

from helpers import mixed_workload, oracle_grid, oracle_params, relerr

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 1e-4
SCHEMES = {"euler": pf.PF_EULER, "heun": pf.PF_HEUN}


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pf.lib()


def oracle_ex(w, steps, scheme, every, rtol=None):
    return O.step_ex(oracle_grid(w), oracle_params(w, rtol), w.P0, None, steps, scheme, every, 0)


def gpu_ex(w, chunks, scheme, every, **over):
    f = Film(w, integrator=SCHEMES[scheme], poisson_every=every, **over)
    infos = [f.step(c)[1] for c in chunks]
    P, phi = f.numpy()
    f.close()
    return P, phi, infos


@pytest.mark.parametrize("scheme,every,solver,eps", [
    ("heun", 1, "pcg", False),
    ("heun", 1, "pcg", True),
    ("heun", 1, "mg", False),
    ("euler", 3, "pcg", False),
    ("euler", 5, "mg", False),
    ("heun", 2, "pcg", True),
])
def test_fp64_matches_oracle(scheme, every, solver, eps):
    """Ragged grid, random electrode masks and voltages; the steps are split
    over two calls, so the solve schedule must carry over between calls."""
    nx, ny, nz = (40, 24, 12) if solver == "mg" else (37, 22, 11)
    w = mixed_workload(nx, ny, nz, 31, eps=eps, steps=9, rtol=1e-13).with_(solver=solver, maxit=3000)
    P, phi, infos = gpu_ex(w, [4, 5], scheme, every)
    Po, phio, sto, io = oracle_ex(w, 9, scheme, every, rtol=1e-14)
    assert sto == O.OK
    assert relerr(P, Po) <= FP64_TOL
    assert relerr(phi, phio) <= FP64_TOL
    solves = sum(1 for n in range(9) if n % every == 0) * (2 if scheme == "heun" else 1)
    assert all(i["status"] == pf.PF_OK for i in infos)
    assert sum(i["graph_steps"] for i in infos) == 9
    assert sum(i["total_iters"] for i in infos) >= solves


def test_heun_fp32_strips_vs_fp64_oracle():
    w = W.film_strip_fp32(64, 64, 16, steps=40)
    P, phi, infos = gpu_ex(w, [40], "heun", 1)
    Po, phio, sto, _ = oracle_ex(w, 40, "heun", 1, rtol=1e-12)
    assert sto == O.OK
    assert relerr(P, Po) <= FP32_TOL


def test_heun_graph_and_host_driven_agree():
    """Graph-launched and host-driven (profiling on) steps of the predictor-
    corrector with a solve every 2 steps give bit-identical states."""
    w = mixed_workload(48, 32, 8, 43, precision="fp32", steps=5, rtol=1e-7).with_(solver="mg", maxit=500)
    res = []
    for prof in (0, 1):
        f = Film(w, integrator=pf.PF_HEUN, poisson_every=2)
        if prof:
            pf.pf_profile_enable(f.ctx, 1)
        _, info = f.step(5)
        res.append((f.numpy(), info))
        f.close()
    (a, ia), (b, ib) = res
    assert ia["graph_steps"] == 5 and ib["graph_steps"] == 0
    assert ia["total_iters"] == ib["total_iters"]
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_heun_is_second_order_in_time_on_the_gpu():
    """Against a 4x finer predictor-corrector run, halving dt cuts the error by
    about 4 (forward Euler: about 2): the corrector is applied as stated."""
    base = mixed_workload(24, 16, 8, 47, steps=1, rtol=1e-13)
    T = 0.4

    def run(scheme, dt):
        w = base.with_(dt=dt, steps=int(round(T / dt)))
        P, _, _ = gpu_ex(w, [w.steps], scheme, 1)
        return P

    ref = run("heun", 0.005)
    for scheme, ratio in (("heun", 4.0), ("euler", 2.0)):
        e1 = np.abs(run(scheme, 0.04) - ref).max()
        e2 = np.abs(run(scheme, 0.02) - ref).max()
        assert e1 / e2 == pytest.approx(ratio, rel=0.25)


def test_adjoint_rejects_other_integrators():
    w = mixed_workload(16, 16, 8, 5, steps=1)
    f = Film(w, integrator=pf.PF_HEUN, flags=pf.PF_FLAG_ADJOINT)
    lam = torch.zeros_like(f.P)
    out = torch.zeros_like(f.P)
    grad = torch.zeros(4, dtype=torch.float64, device=f.P.device)
    with pytest.raises(pf.PfError) as e:
        pf.pf_adjoint_step(f.ctx, lam, out, grad)
    assert e.value.status == pf.PF_ERR_NOTIMPL
    f.close()
