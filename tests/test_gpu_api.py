"""Entry points around the step: the asynchronous step pair, the FP64 true
residual, the host-resident step, and the compensated FP32 polarization
state, checked through the C ABI against pf_step, the FP64 oracle and the
FP64 GPU path (itself pinned to the oracle)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1202_6116_gb300 import build as B
from paper_1202_6116_gb300 import pf
from paper_1202_6116_gb300 import workloads as W
from paper_1202_6116_gb300.film import Film

from helpers import mixed_workload, oracle_grid, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pf.lib()


@pytest.mark.parametrize("solver", ["pcg", "mg"])
def test_step_async_matches_step(solver):
    """Three asynchronous calls then one wait give bit for bit the state of
    one pf_step call over the same steps, and the same statistics."""
    w = W.film_tip_fp32(64, 64, 16, seed=2).with_(solver=solver, maxit=500 if solver == "mg" else 3000)
    a = Film(w)
    st_a, ia = a.step(7)
    b = Film(w)
    b.step_async(2)
    b.step_async(3)
    b.step_async(2)
    st_b, ib = b.wait()
    assert st_a == st_b == pf.PF_OK
    assert torch.equal(a.P, b.P) and torch.equal(a.phi, b.phi)
    for k in ("steps_done", "total_iters", "last_iters", "max_iters", "solves", "nonconverged"):
        assert ia[k] == ib[k], k
    assert ib["solves"] == 7 and ib["max_iters"] >= ib["last_iters"]
    a.close()
    b.close()


def test_pending_async_work_blocks_other_calls():
    w = mixed_workload(16, 8, 4, 40, steps=2)
    f = Film(w)
    f.step_async(2)
    for call in (lambda: f.solve_potential(), lambda: f.diagnostics(), lambda: f.true_residual(),
                 lambda: pf.pf_step_host(f.ctx, f.P.cpu().pin_memory(), f.phi.cpu().pin_memory(), 1)):
        with pytest.raises(pf.PfError) as e:
            call()
        assert e.value.status == pf.PF_ERR_STATE
    st, info = f.step(1)                 # pf_step joins the pending work
    assert st == pf.PF_OK and info["steps_done"] == 3
    st, info = f.wait()                  # nothing pending: an empty report
    assert info["steps_done"] == 0 and info["solves"] == 0
    f.close()


def numpy_residual(w, P, phi):
    G = oracle_grid(w)
    b = O.rhs(G, P)
    if not O.has_dirichlet(G):
        b = b - b.mean()
    r = b - O.apply(G, phi)
    return np.sqrt((r * r).sum()), np.sqrt((b * b).sum())


@pytest.mark.parametrize("precision,eps,singular", [("fp64", False, False), ("fp64", True, False),
                                                    ("fp32", False, False), ("fp64", False, True)])
def test_true_residual_matches_the_oracle_operators(precision, eps, singular):
    """||b(P) - A phi|| and ||b(P)|| for an arbitrary (P, phi): the FP64
    device computation against the oracle's right-hand side and operator on
    the same stored values (FP32 values widened exactly to FP64)."""
    w = mixed_workload(24, 20, 10, 41, precision=precision, eps=eps, tol_dirichlet=0.0 if singular else 0.5)
    if singular:
        w = w.with_(type_lo=np.zeros_like(w.type_lo), type_hi=np.zeros_like(w.type_hi))
    if precision == "fp32":               # the device holds the face voltages in the field precision
        w = w.with_(volt_lo=w.volt_lo.astype(np.float32).astype(np.float64),
                    volt_hi=w.volt_hi.astype(np.float32).astype(np.float64))
    f = Film(w)
    rng = np.random.default_rng(5)
    phi = rng.uniform(-1, 1, w.shape)
    f.phi.copy_(torch.as_tensor(phi, dtype=f.dtype))
    res, bn, resc = f.true_residual()
    Pst, phist = f.numpy()                 # the stored (possibly FP32) values, widened
    res_o, bn_o = numpy_residual(w, Pst, phist)
    assert res == pytest.approx(res_o, rel=1e-12)
    assert bn == pytest.approx(bn_o, rel=1e-12)
    assert resc == res                     # no compensated history after a bind
    # with an explicit state pointer
    P2 = torch.as_tensor(rng.uniform(-0.5, 0.5, (3,) + w.shape), dtype=f.dtype, device="cuda")
    res2, bn2, _ = f.true_residual(P2)
    res2_o, bn2_o = numpy_residual(w, P2.double().cpu().numpy(), phist)
    assert res2 == pytest.approx(res2_o, rel=1e-12) and bn2 == pytest.approx(bn2_o, rel=1e-12)
    f.close()


def test_true_residual_of_a_converged_solve():
    w = mixed_workload(32, 16, 8, 42, precision="fp64", rtol=1e-12)
    f = Film(w)
    st, info = f.solve_potential()
    res, bn, _ = f.true_residual()
    assert res / bn < 1e-11
    assert info["last_relres"] < 1e-12
    f.close()


def test_true_residual_of_the_compensated_fp32_potential():
    """After FP32 steps with the extrapolated start, the stored FP32 phi is
    the solution rounded to FP32; its true residual is limited by that
    rounding, while the compensated potential (phi plus the kept remainder)
    carries the solve's own accuracy, within a small factor of the tolerance
    (the solver stops on its recursive residual)."""
    w = W.film_tip_fp32(128, 128, 32, seed=2).with_(rtol=1e-7)
    f = Film(w)
    f.step(8)
    Pprev = f.P.clone()
    _, info = f.step(1)
    res, bn, resc = f.true_residual(Pprev)
    print("true relres: stored %.3e, compensated %.3e, recursive %.3e" % (res / bn, resc / bn, info["last_relres"]))
    assert info["last_relres"] < 1e-7
    assert resc / bn < 1e-6
    assert resc < res
    f.close()


def test_step_host_needs_no_device_copy_and_matches():
    """pf_step_host over an odd number of steps (the state ends in the
    workspace copy between steps) equals pf_step bit for bit, FP32 with the
    compensated state."""
    w = W.film_strip_fp32(32, 32, 16, seed=1)
    a = Film(w)
    a.step(5)
    b = Film(w)
    Ph = b.P.detach().cpu().pin_memory()
    phih = b.phi.detach().cpu().pin_memory()
    st, info = pf.pf_step_host(b.ctx, Ph, phih, 5)
    assert st == pf.PF_OK and info.steps_done == 5
    assert torch.equal(Ph, a.P.cpu()) and torch.equal(phih, a.phi.cpu())
    assert torch.equal(b.P, a.P)
    a.close()
    b.close()


def fp64_reference(w, steps):
    f = Film(w.with_(precision="fp64"))
    f.step(steps)
    P = f.P.clone()
    f.close()
    return P


def test_compensated_fp32_state_tracks_fp64():
    """FP32 forward Euler keeps P as an FP32 pair (value + remainder): over a
    long run on the strip film it stays closer to the FP64 path (pinned to
    the oracle by the parity tests) than the plain FP32 state, and within the
    FP32 bar of 1e-4."""
    steps = 1500
    w = W.film_strip_fp32(64, 64, 16, seed=1).with_(solver="mg", maxit=500)
    ref = fp64_reference(w, steps)
    errs = {}
    for key, flags in (("comp", 0), ("plain", pf.PF_FLAG_PLAIN_FP32)):
        f = Film(w, flags=flags)
        f.step(steps)
        errs[key] = max(float((f.P[c].double() - ref[c]).abs().max() / ref[c].abs().max()) for c in range(3))
        f.close()
    print("max rel err of P after %d steps: compensated %.3e, plain %.3e" % (steps, errs["comp"], errs["plain"]))
    assert errs["comp"] <= 1e-4
    assert errs["comp"] <= errs["plain"]


def test_compensated_state_starts_like_the_plain_one():
    """The remainder starts at zero: the first step of both states gives the
    same FP32 values (the pair's leading part is the plainly rounded sum)."""
    w = W.film_strip_fp32(32, 32, 16, seed=1).with_(solver="mg", maxit=500)
    a = Film(w)
    a.step(1)
    b = Film(w, flags=pf.PF_FLAG_PLAIN_FP32)
    b.step(1)
    assert torch.equal(a.phi, b.phi)
    assert relerr(a.P.double().cpu().numpy(), b.P.double().cpu().numpy()) <= 1e-6
    a.close()
    b.close()


@pytest.mark.parametrize("solver", ["pcg", "mg"])
def test_persistent_step_loop_matches_single_steps(solver):
    """A 10-step call runs as one graph launch (pairs of steps in a
    device-counted while loop); ten one-step calls run ten step graphs, and
    host-issued steps run the same kernels: all three give the same state bit
    for bit, and the loop reports every step as graph-run."""
    w = W.film_tip_fp32(64, 64, 16, seed=2).with_(solver=solver, maxit=500 if solver == "mg" else 3000)
    a = Film(w)
    st, ia = a.step(10)
    assert st == pf.PF_OK and ia["graph_steps"] == 10 and ia["solves"] == 10
    b = Film(w)
    for _ in range(10):
        b.step(1)
    c = Film(w, flags=pf.PF_FLAG_NO_GRAPHS)
    c.step(10)
    assert torch.equal(a.P, b.P) and torch.equal(a.phi, b.phi)
    assert torch.equal(a.P, c.P) and torch.equal(a.phi, c.phi)
    for f in (a, b, c):
        f.close()
