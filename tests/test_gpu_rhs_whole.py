"""The whole-tile kernels of an FP32 time series on 64 x 16 tiles -- the
Poisson right-hand side and warm residual (k_rhs_w: each field staged with
only the neighbours its term reads) and the compensated TDGL update
(k_tdgl_w: the halo copies spread over the block) -- against the FP64 oracle,
and against the general plane march (vx = 1 tiling) on the same films:
electrode masks and voltages on both z faces, a singular periodic box
(zero-mean b), and tilings one plane deep, a whole film deep and with one
block per SM."""
import numpy as np
import pytest
import torch

from paper_1202_6116_gb300 import build as B
from paper_1202_6116_gb300 import pf
from paper_1202_6116_gb300 import workloads as W
from paper_1202_6116_gb300.film import Film

from helpers import mixed_workload, oracle_run, relerr

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4
AGREE = 1e-5          # two FP32 runs whose sums are formed in another order


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pf.lib()


def run(w, tiling=None, steps=None):
    f = Film(w)
    if tiling is not None:
        pf.pf_set_tiling(f.ctx, *tiling)
    st, info = f.step(w.steps if steps is None else steps)
    assert st == pf.PF_OK
    P, phi = f.numpy()
    f.close()
    return P, phi, info


def mixed32(nx=128, ny=64, nz=12, seed=11):
    return mixed_workload(nx, ny, nz, seed, precision="fp32", steps=8, rtol=1e-7)


@pytest.mark.parametrize("solver", ["pcg", "mg"])
def test_whole_tiles_vs_oracle_and_general_march(solver):
    w = mixed32().with_(solver=solver, maxit=3000 if solver == "pcg" else 300)
    Po, phio, _, _ = oracle_run(w.with_(precision="fp64"), rtol=1e-12)
    P, phi, _ = run(w)
    assert relerr(P, Po) <= FP32_TOL and relerr(phi, phio) <= FP32_TOL
    Pg, phig, _ = run(w, tiling=(1, 4, 0))          # vx = 1: the general kernel
    assert relerr(P, Pg) <= AGREE and relerr(phi, phig) <= AGREE


def test_whole_tiles_singular_periodic_box():
    """No electrode, periodic z: b is projected to zero mean before the
    residual (the mean is subtracted in the whole-tile kernel)."""
    nx, ny, nz = 64, 32, 12
    z8 = np.zeros((ny, nx), np.int8)
    zv = np.zeros((ny, nx))
    w = W.Workload("singular", nx, ny, nz, W.random_film(nx, ny, nz, 5, -0.5, 0.5), z8, zv, z8, zv,
                   periodic_z=True, steps=6, rtol=1e-7, precision="fp32")
    Po, phio, _, _ = oracle_run(w.with_(precision="fp64"), rtol=1e-12)
    P, phi, _ = run(w)
    assert abs(float(phi.mean())) < 1e-6 * max(1.0, float(np.abs(phi).max()))
    assert relerr(P, Po) <= FP32_TOL and relerr(phi, phio) <= FP32_TOL


@pytest.mark.parametrize("tiling", [(4, 1, 0), (4, 64, 0), (4, 3, 1)])
def test_whole_tiles_any_depth_and_grid(tiling):
    """Tiles one plane deep (every plane a tile's first and last), one tile
    over the whole depth, a ragged depth with one block per SM: the same
    state as the default tiling up to the order of the sums."""
    w = mixed32(nz=13, seed=12)
    P, phi, _ = run(w)
    Pt, phit, _ = run(w, tiling=tiling)
    assert relerr(Pt, P) <= AGREE and relerr(phit, phi) <= AGREE


@pytest.mark.parametrize("shape", [(64, 16, 1), (64, 16, 2), (128, 32, 3)])
def test_whole_tiles_thin_films(shape):
    """One tile column and row (the x and y halo wrap onto the tile itself),
    one plane touching both z faces, two planes, three: against the oracle
    and against the general march."""
    nx, ny, nz = shape
    w = mixed_workload(nx, ny, nz, 73, precision="fp32", steps=4, rtol=1e-7, amp=0.5)
    Po, phio, _, _ = oracle_run(w.with_(precision="fp64"), rtol=1e-14)
    P, phi, _ = run(w)
    assert relerr(P, Po) <= FP32_TOL and relerr(phi, phio) <= 1e-3
    Pg, phig, _ = run(w, tiling=(1, 4, 0))
    assert relerr(P, Pg) <= AGREE and relerr(phi, phig) <= 10 * AGREE
