"""Pins of the oracle's discrete adjoint against things other than itself.

The adjoint of the forward-Euler TDGL + Poisson step (Eqs. TDGL, rho, Poisson;
Section Time Integration) is pinned by
  * central finite differences of the oracle's own forward map (brute force:
    every derivative of a scalar J = <w, P_S> with respect to the initial
    state, the four coefficients and the electrode voltages);
  * the symmetry of the one-step Jacobian that the derivation rests on
    (the face rules make the field operator the transpose of the divergence),
    checked as <u, J^T v> = <J^T u, v> for random u, v.
Cases cover mixed electrodes with a permittivity field, a spacing dx != 1,
the all-Neumann (singular) box and a z-periodic box.  The forward solves run
at rtol 1e-14 so the finite differences see an exact Poisson solve.
"""
import numpy as np
import pytest

import oracle
from paper_1202_6116_gb300.workloads import uniform


def _case(kind):
    nx, ny, nz = 6, 5, 4
    m = (ny, nx)
    tl = np.zeros(m, np.int8)
    th = np.zeros(m, np.int8)
    vl = np.zeros(m)
    vh = np.zeros(m)
    eps = None
    dx = 1.0
    periodic = False
    if kind in ("mixed", "dx"):
        th[:, 1:3] = 1
        vh[:, 1:3] = 0.7
        th[:, 4] = 1
        vh[:, 4] = -0.4
        tl[1:4, :] = 1
        vl[1:4, :] = 0.25 * (uniform(11, nx * 3).reshape(3, nx) - 0.5)
        eps = 1.0 + 3.0 * uniform(12, nx * ny * nz).reshape(nz, ny, nx)
        if kind == "dx":
            dx = 0.7
    elif kind == "periodic":
        periodic = True
    G = oracle.Grid(nx, ny, nz, dx=dx, periodic_z=periodic, type_lo=tl, volt_lo=vl, type_hi=th,
                    volt_hi=vh, eps=eps)
    prm = oracle.Params(a1=-1.0, a11=0.5, a12=0.8, g=0.5, L=1.0, dt=0.02, rtol=1e-14)
    P0 = 0.8 * (uniform(13, 3 * nx * ny * nz).reshape((3,) + G.shape) - 0.5)
    w = uniform(14, 3 * nx * ny * nz).reshape((3,) + G.shape) - 0.5
    return G, prm, P0, w


NSTEPS = 3


def _J(G, prm, P0, w):
    P, _phi, st, _ = oracle.step(G, prm, P0, None, NSTEPS)
    assert st == oracle.OK
    return float(np.sum(w * P))


def _fd(f, h):
    return (f(h) - f(-h)) / (2.0 * h)


def _close(a, b, tol):
    return abs(a - b) <= tol * max(abs(b), 1e-30)


@pytest.mark.parametrize("kind", ["mixed", "dx", "neumann", "periodic"])
def test_adjoint_matches_finite_differences(kind):
    G, prm, P0, w = _case(kind)
    lam0, grad, gv_lo, gv_hi = oracle.gradient(G, prm, P0, w, NSTEPS)

    # initial state, along a random direction
    v = uniform(15, P0.size).reshape(P0.shape) - 0.5
    d = _fd(lambda h: _J(G, prm, P0 + h * v, w), 1e-5)
    assert _close(float(np.sum(lam0 * v)), d, 1e-7), (np.sum(lam0 * v), d)

    # Landau coefficients and the gradient coefficient
    for k, name in enumerate(["a1", "a11", "a12", "g"]):
        base = getattr(prm, name)

        def f(h, name=name, base=base):
            p = oracle.Params(**{**prm.__dict__, name: base + h})
            return _J(G, p, P0, w)

        d = _fd(f, 1e-5)
        assert _close(grad[k], d, 1e-7), (name, grad[k], d)

    # electrode voltages, along a random direction over the Dirichlet cells
    if kind in ("mixed", "dx"):
        ulo = (uniform(16, G.nx * G.ny).reshape(G.ny, G.nx) - 0.5) * (G.type_lo == 1)
        uhi = (uniform(17, G.nx * G.ny).reshape(G.ny, G.nx) - 0.5) * (G.type_hi == 1)

        def fv(h):
            Gh = oracle.Grid(G.nx, G.ny, G.nz, dx=G.dx, type_lo=G.type_lo, volt_lo=G.volt_lo + h * ulo,
                             type_hi=G.type_hi, volt_hi=G.volt_hi + h * uhi, eps=G.eps)
            return _J(Gh, prm, P0, w)

        d = _fd(fv, 1e-5)
        a = float(np.sum(gv_lo * ulo) + np.sum(gv_hi * uhi))
        assert _close(a, d, 1e-7), (a, d)
        # a Neumann face cell has no voltage to differentiate
        assert np.all(gv_lo[G.type_lo == 0] == 0.0) and np.all(gv_hi[G.type_hi == 0] == 0.0)
        # both faces carry sensitivity somewhere
        assert np.abs(gv_lo).max() > 0 and np.abs(gv_hi).max() > 0


@pytest.mark.parametrize("kind", ["mixed", "neumann", "periodic"])
def test_one_step_jacobian_is_symmetric(kind):
    G, prm, P0, _w = _case(kind)
    u = uniform(21, P0.size).reshape(P0.shape) - 0.5
    v = uniform(22, P0.size).reshape(P0.shape) - 0.5
    Ju = oracle.adjoint_step(G, prm, P0, u)[0]
    Jv = oracle.adjoint_step(G, prm, P0, v)[0]
    a, b = float(np.sum(Ju * v)), float(np.sum(u * Jv))
    assert abs(a - b) <= 1e-12 * max(abs(a), 1.0)


def test_adjoint_is_linear_in_lambda_and_zero_for_zero():
    G, prm, P0, w = _case("mixed")
    out, psi, grad, glo, ghi, st, it = oracle.adjoint_step(G, prm, P0, np.zeros_like(P0))
    assert st == oracle.OK and it == 0
    assert np.all(out == 0) and np.all(grad == 0) and np.all(glo == 0) and np.all(ghi == 0)
    a = oracle.adjoint_step(G, prm, P0, w)
    b = oracle.adjoint_step(G, prm, P0, 2.0 * w)
    assert np.allclose(b[0], 2.0 * a[0], rtol=1e-12, atol=1e-14)
    assert np.allclose(b[2], 2.0 * a[2], rtol=1e-12, atol=1e-14)
