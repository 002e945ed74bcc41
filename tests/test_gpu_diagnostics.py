"""GPU run diagnostics (pf_diagnostics) against the oracle's definitions on
the same state, and the discrete free energy decreasing along GPU steps."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1202_6116_gb300 import build as B
from paper_1202_6116_gb300 import pf
from paper_1202_6116_gb300 import workloads as W
from paper_1202_6116_gb300.film import Film

from helpers import mixed_workload, oracle_grid, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pf.lib()


def _compare(f, w, tol, thr=0.3):
    P, phi = f.numpy()
    d = f.diagnostics(thr)
    o = O.diagnostics(oracle_grid(w), oracle_params(w), P, phi, thr)
    assert d["switched_fraction"] == o["switched_fraction"]
    for k in ("mean_px", "mean_py", "mean_pz"):
        assert abs(d[k] - o[k]) <= tol * max(np.abs(P).max(), 1e-30), k
    for k in ("f_landau", "f_grad", "f_elec"):
        assert abs(d[k] - o[k]) <= tol * max(abs(o[k]), 1e-30), (k, d[k], o[k])
    return d


def test_diagnostics_fp64_mixed_electrodes():
    """Ragged 40 x 36 x 12, random electrodes with voltages and eps, after 5 steps."""
    w = mixed_workload(40, 36, 12, seed=51, eps=True, amp=0.7)
    f = Film(w)
    f.step(5)
    f.solve_potential()
    _compare(f, w, 1e-12)
    f.close()


def test_diagnostics_fp32_stripes_and_tip():
    w = W.film_tip_fp32(128, 128, 16, steps=3).with_(solver="pcg", maxit=20000)
    f = Film(w)
    f.step(3)
    d = _compare(f, w, 1e-5)
    assert 0.0 < d["switched_fraction"] < 1.0
    f.close()


def test_diagnostics_periodic_box_and_thresholds():
    w = mixed_workload(32, 16, 8, seed=52).with_(periodic_z=True)
    f = Film(w)
    f.step(2)
    f.solve_potential()
    for thr in (-1.0, 0.0, 0.3, 2.0):
        _compare(f, w, 1e-12, thr)
    assert f.diagnostics(-1.0)["switched_fraction"] == 1.0
    assert f.diagnostics(2.0)["switched_fraction"] == 0.0
    f.close()


def test_free_energy_decreases_along_gpu_steps():
    """Electrodes at 0 V: F = f_landau + f_grad + f_elec of each state (phi
    solved for that state) falls at every step."""
    w = mixed_workload(32, 32, 8, seed=53, eps=True, volts=False, amp=0.6, rtol=1e-13)
    f = Film(w)
    F = []
    for _ in range(15):
        f.solve_potential()
        d = f.diagnostics()
        F.append(d["f_landau"] + d["f_grad"] + d["f_elec"])
        f.step(1)
    f.close()
    assert all(b < a for a, b in zip(F, F[1:])), F
