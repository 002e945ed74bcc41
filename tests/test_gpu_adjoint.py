"""GPU parity of the discrete adjoint (pf_adjoint_step) and of gradients
taken through it.

  * each adjoint step against the oracle's adjoint step on the same state,
    cotangent and warm start (FP64: 1e-10 normwise on lam, the coefficient
    gradients and the face-voltage gradients; FP32: 1e-4);
  * whole-trajectory gradients (torch.autograd through the adjoint with
    checkpoint-and-recompute) against central finite differences of the GPU
    forward map, step 1e-6, forward solves at rtol 1e-14: <= 1e-6 relative,
    for a1, a11, a12, g, both strip-electrode voltages and the initial state.
The loss is the mean-squared difference between the final P_z and a target
made by the same model with a11 = 0.55 and the electrodes at +-2.2.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1202_6116_gb300 import build as B
from paper_1202_6116_gb300 import pf
from paper_1202_6116_gb300 import workloads as W
from paper_1202_6116_gb300.adjoint import TrajectorySpec, final_state, trajectory
from paper_1202_6116_gb300.film import Film

from helpers import mixed_workload, oracle_grid, oracle_params, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pf.lib()


def _vec_relerr(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def _adjoint_chain(w, nsteps, tol, seed=7, **over):
    """Oracle forward states P_0..P_{n-1}; then n adjoint steps backwards on
    both sides from the same random cotangent, compared after every step."""
    G, prm = oracle_grid(w), oracle_params(w, rtol=1e-14)
    prm.maxit = 100000
    states = [np.array(w.P0, dtype=np.float64)]
    phi = None
    for _ in range(nsteps - 1):
        P, phi, st, _ = O.step(G, prm, states[-1], phi, 1)
        assert st == O.OK
        states.append(P)
    lam0 = W.uniform(seed, 3 * w.n).reshape((3,) + w.shape) - 0.5
    f = Film(w, flags=pf.PF_FLAG_ADJOINT, **over)
    dt = f.dtype
    lam = torch.as_tensor(lam0, dtype=dt, device="cuda").contiguous()
    lam_out = torch.empty_like(lam)
    grad = torch.zeros(4, dtype=torch.float64, device="cuda")
    gv = torch.zeros((2, w.ny, w.nx), dtype=torch.float64, device="cuda")
    o_lam, o_psi = lam0.copy(), None
    o_grad, o_glo, o_ghi = np.zeros(4), np.zeros((w.ny, w.nx)), np.zeros((w.ny, w.nx))
    iters = []
    for k in range(nsteps - 1, -1, -1):
        f.P.copy_(torch.as_tensor(states[k], dtype=dt, device="cuda"))
        st, info = pf.pf_adjoint_step(f.ctx, lam, lam_out, grad, gv)
        assert st == pf.PF_OK
        iters.append(info.last_iters)
        lam, lam_out = lam_out, lam
        o_lam, o_psi, g4, glo, ghi, ost, _ = O.adjoint_step(G, prm, states[k], o_lam, o_psi)
        assert ost == O.OK
        o_grad += g4
        o_glo += glo
        o_ghi += ghi
        assert relerr(lam.double().cpu().numpy(), o_lam) <= tol, k
        assert _vec_relerr(grad.cpu().numpy(), o_grad) <= tol, (k, grad.cpu().numpy(), o_grad)
        gvh = gv.cpu().numpy()
        if np.abs(o_glo).max() > 0:
            assert relerr(gvh[0], o_glo) <= tol
        else:
            assert np.all(gvh[0] == 0)
        if np.abs(o_ghi).max() > 0:
            assert relerr(gvh[1], o_ghi) <= tol
        else:
            assert np.all(gvh[1] == 0)
    f.close()
    return iters


def test_adjoint_steps_fp64_mixed_electrodes_with_eps():
    """Ragged 40 x 36 x 12 grid (several tiles, partial last tile), random
    Dirichlet/Neumann face cells with voltages, a permittivity field."""
    w = mixed_workload(40, 36, 12, seed=31, eps=True, rtol=1e-14)
    _adjoint_chain(w, 3, 1e-10)


def test_adjoint_steps_fp64_singular_box():
    """No electrode anywhere: the adjoint solve is singular (zero-mean gauge)."""
    nx, ny, nz = 32, 24, 10
    P0 = W.random_film(nx, ny, nz, 32, -0.5, 0.5)
    z8, zv = np.zeros((ny, nx), np.int8), np.zeros((ny, nx))
    w = W.Workload("neumann", nx, ny, nz, P0, z8, zv, z8.copy(), zv.copy(), rtol=1e-14)
    _adjoint_chain(w, 2, 1e-10)


def test_adjoint_steps_fp64_multigrid():
    w = W.film_adjoint_fp64(64, 64, 16).with_(solver="mg", rtol=1e-13, maxit=300)
    _adjoint_chain(w, 2, 1e-10)


def test_adjoint_steps_fp32():
    w = W.film_adjoint_fp64(64, 64, 16).with_(precision="fp32", rtol=1e-8)
    _adjoint_chain(w, 2, 1e-4)


def test_adjoint_argument_checks():
    w = W.film_adjoint_fp64(32, 32, 8)
    f = Film(w)                                   # no PF_FLAG_ADJOINT
    lam = torch.zeros((3,) + w.shape, dtype=torch.float64, device="cuda")
    out = torch.empty_like(lam)
    grad = torch.zeros(4, dtype=torch.float64, device="cuda")
    st, _ = pf.pf_adjoint_step(f.ctx, lam, out, grad, None, ok=(pf.PF_ERR_STATE,))
    assert st == pf.PF_ERR_STATE
    f.close()
    f = Film(w, flags=pf.PF_FLAG_ADJOINT)
    st, _ = pf.pf_adjoint_step(f.ctx, lam, lam, grad, None, ok=(pf.PF_ERR_ARG,))
    assert st == pf.PF_ERR_ARG                    # lam_out overlaps lam_in
    st, _ = pf.pf_adjoint_step(f.ctx, lam, f.P, grad, None, ok=(pf.PF_ERR_ARG,))
    assert st == pf.PF_ERR_ARG                    # lam_out overlaps the bound P
    st, _ = pf.pf_adjoint_step(f.ctx, lam, out, None, None, ok=(pf.PF_ERR_ARG,))
    assert st == pf.PF_ERR_ARG
    host = torch.zeros(4, dtype=torch.float64)
    st, _ = pf.pf_adjoint_step(f.ctx, lam, out, host, None, ok=(pf.PF_ERR_ARG,))
    assert st == pf.PF_ERR_ARG                    # gradients live on the device
    # a zero cotangent gives a zero adjoint and adds nothing
    st, info = pf.pf_adjoint_step(f.ctx, lam, out, grad, None)
    assert st == pf.PF_OK and info.last_iters == 0
    assert torch.count_nonzero(out).item() == 0 and torch.count_nonzero(grad).item() == 0
    f.close()


# ------------------------------------------------------------- trajectories

def _strip_masks(w):
    plus = (w.type_hi == 1) & (w.volt_hi > 0)
    minus = (w.type_hi == 1) & (w.volt_hi < 0)
    return plus, minus


def _c3_problem(nx, ny, nz, steps, K, solver="pcg"):
    w = W.film_adjoint_fp64(nx, ny, nz, steps=steps).with_(rtol=1e-14, solver=solver,
                                                          maxit=500 if solver == "mg" else 20000)
    plus, minus = _strip_masks(w)
    spec = TrajectorySpec(w, steps=steps, checkpoint_every=K)
    vlo = torch.zeros(w.ny, w.nx, dtype=torch.float64)
    mp = torch.as_tensor(plus, dtype=torch.float64)
    mm = torch.as_tensor(minus, dtype=torch.float64)
    target = final_state(spec, [w.a1, 0.55, w.a12, w.g], vlo, 2.2 * mp - 2.2 * mm)[2]
    return w, spec, vlo, mp, mm, target


def _loss_fd(spec, target, theta, P0=None):
    a1, a11, a12, g, vp, vm = theta
    vlo = torch.zeros(spec.workload.ny, spec.workload.nx, dtype=torch.float64)
    plus, minus = _strip_masks(spec.workload)
    vhi = vp * torch.as_tensor(plus, dtype=torch.float64) + vm * torch.as_tensor(minus, dtype=torch.float64)
    P = final_state(spec, [a1, a11, a12, g], vlo, vhi, P0=P0)
    return float(((P[2] - target) ** 2).mean())


def _check_gradients(nx, ny, nz, steps, K, tol=1e-6, h=1e-6, solver="pcg"):
    w, spec, vlo, mp, mm, target = _c3_problem(nx, ny, nz, steps, K, solver)
    P0 = torch.as_tensor(np.ascontiguousarray(w.P0), device="cuda").requires_grad_(True)
    theta0 = [w.a1, w.a11, w.a12, w.g, 2.0, -2.0]
    coeffs = torch.tensor(theta0[:4], dtype=torch.float64, requires_grad=True)
    v = torch.tensor(theta0[4:], dtype=torch.float64, requires_grad=True)
    vhi = v[0] * mp + v[1] * mm
    P = trajectory(P0, coeffs, vlo, vhi, spec)
    loss = ((P[2] - target) ** 2).mean()
    loss.backward()
    adj = list(coeffs.grad.numpy()) + list(v.grad.numpy())
    for k in range(6):
        tp, tm = list(theta0), list(theta0)
        tp[k] += h
        tm[k] -= h
        fd = (_loss_fd(spec, target, tp) - _loss_fd(spec, target, tm)) / (2 * h)
        assert abs(adj[k] - fd) <= tol * abs(fd), (k, adj[k], fd)
    d = torch.as_tensor(W.uniform(41, 3 * w.n).reshape((3,) + w.shape) - 0.5, device="cuda")
    Pp = P0.detach() + h * d
    Pm = P0.detach() - h * d
    fd = (_loss_fd(spec, target, theta0, Pp) - _loss_fd(spec, target, theta0, Pm)) / (2 * h)
    a = float((P0.grad * d).sum())
    assert abs(a - fd) <= tol * abs(fd), (a, fd)
    return adj


def test_trajectory_gradients_match_finite_differences():
    """128 x 128 x 32 strip-electrode film, 40 steps, checkpoints every 10."""
    _check_gradients(128, 128, 32, 40, 10)


def test_trajectory_gradients_full_differentiation_config():
    """The full differentiation workload: 128 x 128 x 32, 500 steps,
    checkpoint-and-recompute every 50 steps (multigrid-preconditioned CG to
    1e-14 in the forward and adjoint solves)."""
    _check_gradients(128, 128, 32, 500, 50, solver="mg")
