"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, on the
same seeded inputs.  Error metric: max|gpu - oracle| / max|oracle| per field.
FP64 bar 1e-10 on P and phi; FP32 bar 1e-4 on P (FP32 storage, FP64-accurate
Poisson reductions) and the switched fraction within 0.1 percentage points."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1202_6116_gb300 import build as B
from paper_1202_6116_gb300 import pf
from paper_1202_6116_gb300 import workloads as W
from paper_1202_6116_gb300.film import Film

from helpers import mixed_workload, oracle_run, relerr, switched_fraction, oracle_grid

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pf.lib()


def gpu_run(w, steps=None, **over):
    f = Film(w, **over)
    st, info = f.step(w.steps if steps is None else steps, ok=(pf.PF_OK, pf.PF_ERR_NOCONV))
    P, phi = f.numpy()
    f.close()
    return P, phi, st, info


@pytest.fixture(scope="module")
def grounded_32():
    w = W.film_fp64_grounded()
    ref = oracle_run(w)
    ref_tight = oracle_run(w, rtol=1e-14)
    return w, ref, ref_tight


def test_fp64_grounded_film_200_steps(grounded_32):
    """32^3 FP64 film between grounded electrodes, 200 steps at CG 1e-12, each
    solve warm-started from the last potential as in the paper (and in the
    oracle): the same results and about the same Jacobi-PCG iteration count."""
    w, (Po, phio, sto, io), (Pt, phit, _, _) = grounded_32
    P, phi, st, info = gpu_run(w, flags=pf.PF_FLAG_WARM_LAST)
    assert st == pf.PF_OK and sto == O.OK
    assert relerr(P, Po) <= FP64_TOL
    assert relerr(phi, phio) <= FP64_TOL
    assert relerr(P, Pt) <= FP64_TOL
    assert relerr(phi, phit) <= FP64_TOL
    assert abs(info["total_iters"] - io["total_iters"]) <= 0.02 * io["total_iters"] + 5
    assert info["graph_steps"] == w.steps          # every step ran as one CUDA graph


def test_fp64_extrapolated_warm_start(grounded_32):
    """The default start of each step solve extrapolates the last
    potentials: the same results within the solve tolerance, fewer
    iterations than the last-potential start."""
    w, (Po, phio, sto, io), (Pt, phit, _, _) = grounded_32
    P, phi, st, info = gpu_run(w)
    assert st == pf.PF_OK
    assert relerr(P, Pt) <= FP64_TOL
    assert relerr(phi, phit) <= FP64_TOL
    assert info["total_iters"] < 0.8 * io["total_iters"]      # 1e-12 Jacobi-PCG: about 0.72


def test_extrapolation_history_survives_calls_and_resets():
    """Steps split over calls equal one call (the history lives on the device);
    a standalone solve resets it (the next step starts from that potential)."""
    w = mixed_workload(40, 24, 12, 61, steps=8, rtol=1e-13)
    a = Film(w)
    a.step(8)
    Pa, phia = a.numpy()
    a.close()
    b = Film(w)
    b.step(3)
    b.step(5)
    Pb, phib = b.numpy()
    b.close()
    assert np.array_equal(Pa, Pb) and np.array_equal(phia, phib)
    c = Film(w)
    c.step(3)
    c.solve_potential()
    _, ic = c.step(5)
    Pc, _ = c.numpy()
    c.close()
    assert relerr(Pc, Pa) <= FP64_TOL and ic["total_iters"] > 0


@pytest.mark.parametrize("precision,rtol,bound", [("fp64", 1e-10, 1e-7), ("fp32", 1e-7, 1e-5)])
def test_extrapolation_is_exact_for_cubic_potentials(precision, rtol, bound):
    """With the mobility at 0 (P frozen) and the top electrode voltages a cubic
    in the step index, the potentials are that cubic too, so the extrapolation
    of the last four starts each solve from the fifth on within a few
    multiples of the tolerance: at most 2 MG-PCG iterations (a quadratic
    extrapolation would start about 1e-2 off; in FP32 so would a start whose
    potential is rounded to FP32, at about 1e-5).  The potential still equals
    the oracle's for the last voltages."""
    w = mixed_workload(32, 24, 12, 71, steps=1, rtol=rtol, precision=precision).with_(L=0.0, solver="mg", maxit=500)
    volts = [w.volt_hi * (1 + 0.3 * k - 0.05 * k ** 2 + 0.01 * k ** 3) for k in range(10)]
    P0 = w.P0.astype(np.float32).astype(np.float64) if precision == "fp32" else w.P0
    its = {}
    for flags in (0, pf.PF_FLAG_WARM_LAST):
        f = Film(w, flags=flags)
        its[flags] = []
        for v in volts:
            f.set_bc(pf.PF_ZHI, w.type_hi, v)
            _, info = f.step(1)
            its[flags].append(info["last_iters"])
        P, phi = f.numpy()
        f.close()
        assert np.array_equal(P, P0)
    assert max(its[0][4:]) <= 2, its
    assert sum(its[pf.PF_FLAG_WARM_LAST][4:]) >= 2 * max(sum(its[0][4:]), 1), its
    phio, st, _, _ = O.solve_potential(oracle_grid(w.with_(volt_hi=volts[-1])), P0, rtol=1e-14)
    assert st == O.OK and relerr(phi, phio) <= bound


def test_graph_and_host_driven_steps_agree():
    """The same steps launched as CUDA graphs (device-driven Krylov loop) and
    host-driven (profiling on) give bit-identical states."""
    for solver in ("pcg", "mg"):
        w = mixed_workload(48, 32, 8, 41, steps=4, rtol=1e-12).with_(solver=solver, maxit=2000)
        f1 = Film(w)
        st1, i1 = f1.step(4)
        a = f1.numpy()
        f1.close()
        f2 = Film(w)
        pf.pf_profile_enable(f2.ctx, 1)
        st2, i2 = f2.step(4)
        b = f2.numpy()
        f2.close()
        assert i1["graph_steps"] == 4 and i2["graph_steps"] == 0
        assert i1["total_iters"] == i2["total_iters"]
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("case", [
    dict(nx=45, ny=38, nz=13, seed=1, eps=False),
    dict(nx=45, ny=38, nz=13, seed=2, eps=True),
    dict(nx=70, ny=9, nz=3, seed=3, eps=True),
    dict(nx=33, ny=17, nz=1, seed=4, eps=False),
])
def test_fp64_ragged_mixed_boundaries(case):
    """Ragged grids (partial tiles in x, y and z) with random electrode masks and
    voltages on both faces, optionally a random permittivity field."""
    w = mixed_workload(case["nx"], case["ny"], case["nz"], case["seed"], eps=case["eps"], steps=8)
    Po, phio, _, _ = oracle_run(w, rtol=1e-13)
    P, phi, st, _ = gpu_run(w, poisson_rtol=1e-13)
    assert st == pf.PF_OK
    assert relerr(P, Po) <= FP64_TOL
    assert relerr(phi, phio) <= FP64_TOL


@pytest.mark.parametrize("periodic", [True, False])
def test_fp64_singular_problems(periodic):
    """No electrode anywhere: fully periodic box, or open top and bottom.  The
    operator is singular; both sides use the zero-mean potential."""
    nx, ny, nz = 24, 20, 12
    z8 = np.zeros((ny, nx), np.int8)
    zv = np.zeros((ny, nx))
    w = W.Workload("singular", nx, ny, nz, W.random_film(nx, ny, nz, 5, -0.5, 0.5), z8, zv, z8, zv,
                   periodic_z=periodic, steps=6, rtol=1e-13)
    Po, phio, _, _ = oracle_run(w)
    P, phi, st, _ = gpu_run(w)
    assert st == pf.PF_OK
    assert abs(phi.mean()) < 1e-12
    assert relerr(P, Po) <= FP64_TOL
    assert relerr(phi, phio) <= FP64_TOL


def test_fp64_solve_potential_only():
    w = mixed_workload(40, 24, 10, 7, eps=True)
    phio, st, it, rel = O.solve_potential(oracle_grid(w), w.P0, rtol=1e-13)
    f = Film(w, poisson_rtol=1e-13)
    st, info = f.solve_potential()
    P, phi = f.numpy()
    f.close()
    assert st == pf.PF_OK
    assert np.array_equal(P, w.P0)
    assert relerr(phi, phio) <= FP64_TOL
    assert abs(info["last_iters"] - it) <= 2


def test_homogeneous_recurrence_on_gpu():
    """Uniform [111] P between grounded electrodes: phi stays 0, no CG iterations,
    and each component follows p <- p + dt (2p - 5.2 p^3)."""
    nx, ny, nz = 40, 16, 8
    one = np.ones((ny, nx), np.int8)
    zv = np.zeros((ny, nx))
    P0 = np.full((3, nz, ny, nx), 0.1)
    w = W.Workload("uniform", nx, ny, nz, P0, one, zv, one, zv, steps=30, rtol=1e-12)
    P, phi, st, info = gpu_run(w)
    p = 0.1
    for _ in range(30):
        p = p + 0.01 * (2 * p - 5.2 * p ** 3)
    assert st == pf.PF_OK
    assert np.abs(P - p).max() < 1e-15
    assert np.abs(phi).max() == 0.0
    assert info["total_iters"] == 0


def test_noconv_is_reported_and_state_valid():
    w = mixed_workload(32, 16, 8, 9, steps=3, rtol=1e-14)
    # unconverged iterates depend on the initial guess: start from the last potential, as the oracle does
    P, phi, st, info = gpu_run(w, poisson_maxit=2, flags=pf.PF_FLAG_WARM_LAST)
    assert st == pf.PF_ERR_NOCONV
    assert info["nonconverged"] == 3 and info["last_iters"] == 2 and info["steps_done"] == 3
    assert np.isfinite(P).all() and np.isfinite(phi).all()
    Po, phio, sto, io = O.step(oracle_grid(w), O.Params(rtol=1e-14, maxit=2), w.P0, None, 3)
    assert sto == O.NOCONV
    assert relerr(P, Po) <= FP64_TOL and relerr(phi, phio) <= FP64_TOL


def test_nonfinite_input_is_reported():
    w = mixed_workload(16, 16, 4, 10, steps=1)
    w.P0[1, 2, 3, 4] = np.nan
    f = Film(w)
    st, info = f.step(1, ok=(pf.PF_ERR_NONFINITE,))
    f.close()
    assert st == pf.PF_ERR_NONFINITE


def test_step_host_matches_device_path():
    w = mixed_workload(36, 20, 6, 11, steps=4, rtol=1e-12)
    P_dev, phi_dev, _, _ = gpu_run(w)
    f = Film(w)
    Ph = torch.as_tensor(w.P0).clone().pin_memory()
    phih = torch.zeros(w.shape, dtype=torch.float64).pin_memory()
    st, info = pf.pf_step_host(f.ctx, Ph, phih, 4)
    f.close()
    assert st == pf.PF_OK
    assert np.array_equal(Ph.numpy(), P_dev) and np.array_equal(phih.numpy(), phi_dev)


def test_bad_arguments_on_gpu():
    w = mixed_workload(8, 8, 4, 12)
    f = Film(w)
    bad = np.full(64, 3, np.int8)
    with pytest.raises(pf.PfError):
        pf.pf_set_bc(f.ctx, pf.PF_ZLO, bad, None)
    with pytest.raises(pf.PfError):
        pf.pf_set_bc(f.ctx, 5, np.zeros(64, np.int8), None)
    with pytest.raises(pf.PfError):
        pf.pf_bind(f.ctx, f.P, f.phi, None, f.workspace, 16)
    # the failed bind leaves the context unbound: every call reports it
    with pytest.raises(pf.PfError):
        pf.pf_step(f.ctx, 1)
    with pytest.raises(pf.PfError):
        pf.pf_adjoint_step(f.ctx, f.P, f.phi, None, None)
    f.close()


# ------------------------------------------------------------------ FP32 mode

def test_fp32_strip_electrodes_vs_fp64_oracle():
    """The strip-electrode thin film, shrunk to 64x64x16, 100 steps, CG 1e-8:
    FP32 fields with FP64-accurate reductions against the FP64 oracle."""
    w = W.film_strip_fp32(64, 64, 16, steps=100)
    Po, phio, _, _ = oracle_run(w.with_(precision="fp64"), rtol=1e-12)
    P, phi, st, info = gpu_run(w)
    assert st == pf.PF_OK
    assert relerr(P, Po) <= FP32_TOL
    assert abs(switched_fraction(P) - switched_fraction(Po)) <= 1e-3


def test_fp32_tip_electrode_vs_fp64_oracle():
    """The tip-electrode stripe-domain film, shrunk to 64x64x16, 40 steps, CG 1e-7."""
    w = W.film_tip_fp32(64, 64, 16, steps=40).with_(solver="pcg")
    Po, phio, _, _ = oracle_run(w.with_(precision="fp64"), rtol=1e-12)
    P, phi, st, info = gpu_run(w)
    assert st == pf.PF_OK
    assert relerr(P, Po) <= FP32_TOL
    assert abs(switched_fraction(P) - switched_fraction(Po)) <= 1e-3


# ---------------------------------------------------- multigrid-preconditioned CG

@pytest.mark.parametrize("shape", [(32, 32, 32), (48, 40, 8), (64, 32, 6)])
def test_mg_fp64_matches_oracle(shape):
    """MG-PCG (FP64) on grids with full, ragged-tile and semi-coarsened
    hierarchies: the potential solves the same linear system as the oracle's
    Jacobi-PCG, so both agree to the solver tolerance."""
    nx, ny, nz = shape
    w = mixed_workload(nx, ny, nz, 21, steps=5, rtol=1e-13).with_(solver="mg", maxit=300)
    Po, phio, _, _ = oracle_run(w, rtol=1e-13)
    P, phi, st, info = gpu_run(w)
    assert st == pf.PF_OK
    assert relerr(P, Po) <= FP64_TOL
    assert relerr(phi, phio) <= FP64_TOL
    assert info["total_iters"] <= 5 * 40


def test_mg_fp64_grounded_film_200_steps(grounded_32):
    w, (Po, phio, _, _), (Pt, phit, _, _) = grounded_32
    P, phi, st, info = gpu_run(w.with_(solver="mg", maxit=300))
    assert st == pf.PF_OK
    assert relerr(P, Pt) <= FP64_TOL and relerr(phi, phit) <= FP64_TOL
    assert info["total_iters"] < 200 * 25


@pytest.mark.parametrize("periodic", [True, False])
def test_mg_fp64_singular(periodic):
    nx, ny, nz = 32, 16, 8
    z8 = np.zeros((ny, nx), np.int8)
    zv = np.zeros((ny, nx))
    w = W.Workload("singular", nx, ny, nz, W.random_film(nx, ny, nz, 6, -0.5, 0.5), z8, zv, z8, zv,
                   periodic_z=periodic, steps=4, rtol=1e-12, solver="mg", maxit=300)
    Po, phio, _, _ = oracle_run(w, rtol=1e-13)
    P, phi, st, _ = gpu_run(w)
    assert st == pf.PF_OK
    assert abs(phi.mean()) < 1e-12
    assert relerr(P, Po) <= FP64_TOL and relerr(phi, phio) <= 1e-9


@pytest.mark.parametrize("maker", ["tip", "strips"])
def test_mg_fp32_vs_fp64_oracle(maker):
    """FP32 MG-PCG on the shrunk tip-electrode (rtol 1e-7) and strip-electrode
    (rtol 1e-8) films against the FP64 oracle."""
    if maker == "tip":
        w = W.film_tip_fp32(64, 64, 16, steps=40).with_(maxit=300)
    else:
        w = W.film_strip_fp32(64, 64, 16, steps=60).with_(solver="mg", maxit=300)
    Po, phio, _, _ = oracle_run(w.with_(precision="fp64"), rtol=1e-12)
    P, phi, st, info = gpu_run(w)
    assert st == pf.PF_OK
    assert relerr(P, Po) <= FP32_TOL
    assert abs(switched_fraction(P) - switched_fraction(Po)) <= 1e-3
    assert info["total_iters"] <= w.steps * 20


def test_mg_rejects_grids_it_cannot_coarsen():
    from paper_1202_6116_gb300.film import make_params
    w = mixed_workload(45, 38, 13, 1).with_(solver="mg")
    p = make_params(w)
    assert pf.pf_workspace_bytes(p) == 0
    with pytest.raises(pf.PfError):
        pf.pf_create(p, None)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 5, 3), (7, 1, 1), (2, 2, 1), (3, 1, 4), (16, 2, 2)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_degenerate_shapes(shape, precision):
    """Grids one cell thin in any direction (a cell its own x/y neighbour, a
    single plane touching both z faces) against the oracle."""
    nx, ny, nz = shape
    w = mixed_workload(nx, ny, nz, 71, precision=precision, steps=4, rtol=1e-13 if precision == "fp64" else 1e-7,
                       amp=0.5)
    P, phi, st, info = gpu_run(w)
    Po, phio, sto, _ = oracle_run(w, rtol=1e-14)
    assert st == pf.PF_OK and sto == O.OK
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    assert relerr(P, Po) <= tol
    assert relerr(phi, phio) <= (tol if precision == "fp64" else 1e-3)


def test_zero_steps_and_repeated_calls():
    w = mixed_workload(24, 16, 8, 73, steps=3, rtol=1e-13)
    f = Film(w)
    st, info = f.step(0)
    assert st == pf.PF_OK and info["steps_done"] == 0 and info["total_iters"] == 0
    P0, _ = f.numpy()
    assert np.array_equal(P0, w.P0)
    for _ in range(3):
        f.step(1)
    P, phi = f.numpy()
    f.close()
    Po, phio, _, _ = oracle_run(w, rtol=1e-14)
    assert relerr(P, Po) <= FP64_TOL and relerr(phi, phio) <= FP64_TOL
