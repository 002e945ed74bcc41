"""Host-side pieces of the batch and the autotuner (no GPU): the ramp
schedule, the batched-sweep workload recipe, the tiling candidates and the
argument checks of the batch entry points that run before any CUDA call."""
import ctypes as C

import numpy as np
import pytest

from paper_1202_6116_gb300 import autotune as AT
from paper_1202_6116_gb300 import build as B
from paper_1202_6116_gb300 import pf
from paper_1202_6116_gb300 import workloads as W


def test_triangle_wave():
    s = np.array([0.0, 0.125, 0.25, 0.5, 0.75, 0.875, 1.0, 1.25, -0.25, 3.75])
    assert np.allclose(W.tri_wave(s), [0.0, 0.5, 1.0, 0.0, -1.0, -0.5, 0.0, 1.0, -1.0, -1.0], atol=1e-15)
    x = np.linspace(0, 3, 1201)
    y = W.tri_wave(x)
    assert np.abs(y).max() <= 1.0 and np.abs(np.diff(y)).max() <= 4 * (x[1] - x[0]) + 1e-12
    assert W.ramp_volts(2.0, 100.0, 25) == pytest.approx(2.0)
    assert W.ramp_volts(2.0, 100.0, 75) == pytest.approx(-2.0)


def test_batch_hysteresis_recipe():
    d = W.batch_draws()
    assert len(d) == 64 and {s for s, _, _ in d} == set(W.BATCH_SHAPES)
    cells = sum(nx * ny * nz for (nx, ny, nz), _, _ in d)
    assert 1.0e7 < cells < 5.0e7
    assert W.batch_draws(8) == d[:8]                 # counter-based draws: a prefix is stable
    small = ((8, 8, 8), (16, 16, 8), (12, 12, 6), (16, 16, 16))
    a = W.film_batch_hysteresis(shapes=small)
    b = W.film_batch_hysteresis(shapes=small)
    assert len(a) == 64
    assert {(w.nx, w.ny, w.nz) for w in a} == set(small)
    for w, v, (shape, A, T) in zip(a, b, d):
        assert w.extra["ramp"] == (A, T) and (w.nx, w.ny, w.nz) == small[W.BATCH_SHAPES.index(shape)]
        amp, period = w.extra["ramp"]
        assert 1.5 <= amp <= 4.0 and 500.0 <= period <= 2000.0
        assert (w.type_lo == 1).all() and (w.type_hi == 1).all()
        assert w.precision == "fp32" and w.dt == 0.01 and w.rtol == 1e-6 and w.steps == 4000
        assert np.abs(w.P0).max() <= 0.01
        assert np.array_equal(w.P0, v.P0) and w.extra == v.extra
    assert len({w.seed for w in a}) == 64


def test_autotune_candidates():
    w32 = W.film_batch_hysteresis(nfilms=1, shapes=((64, 64, 32),))[0]
    c = AT.candidates(w32)
    assert {t[0] for t in c} == {4, 1}
    assert {t[1] for t in c} == {1, 2, 4, 8, 16, 32}
    w64 = w32.with_(precision="fp64", nz=12)
    c = AT.candidates(w64)
    assert {t[0] for t in c} == {2, 1} and max(t[1] for t in c) == 12
    odd = w32.with_(nx=63)
    assert {t[0] for t in AT.candidates(odd)} == {1}
    assert AT.key_of(w32) == "64x64x32/fp32/pcg/unit"


def test_batch_abi_argument_checks():
    B.build()
    L = pf.lib()
    assert pf.pf_batch_workspace_bytes(0, 10) == 0
    assert pf.pf_batch_workspace_bytes(3, -1) == 0
    small, big = pf.pf_batch_workspace_bytes(3, 0), pf.pf_batch_workspace_bytes(3, 1000)
    assert small > 0 and big >= small + 3 * 4 * 8 * 1000
    out = C.c_void_p()
    assert L.pf_batch_create(None, 2, None, 0, 1, 1, C.byref(out)) == pf.PF_ERR_ARG
    assert out.value is None and pf.pf_batch_last_error(None)
    assert L.pf_batch_step(None, 1, None) == pf.PF_ERR_ARG
    assert L.pf_batch_destroy(None) == pf.PF_OK
    assert L.pf_set_tiling(None, None) == pf.PF_ERR_ARG
