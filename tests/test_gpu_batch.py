"""GPU tests of the film batch (one graph launch per step for many films,
electrode voltage ramps, polarization-voltage loop records), the tiling hook
and the autotuner.  Parity against the FP64 oracle driven step by step with
the same ramp voltages; FP64 bar 1e-10, FP32 1e-4 (as the other parity
tests)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1202_6116_gb300 import autotune as AT
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


def small_batch(precision, shapes=((16, 16, 8), (24, 16, 12), (32, 32, 8)), n=3, seed=7):
    ws = W.film_batch_hysteresis(nfilms=n, seed=seed, steps=12, shapes=shapes, precision=precision, rtol=1e-13)
    # short periods so that a dozen steps sweep through the triangle wave
    return [w.with_(extra={"ramp": (w.extra["ramp"][0], 8.0 + 3 * i)}) for i, w in enumerate(ws)]


def oracle_ramped(w, steps, rtol=1e-14):
    """The oracle stepped one step at a time with the ramp voltage on every
    electrode cell of the top face; returns (P, phi, loop records)."""
    amp, period = w.extra["ramp"]
    G = oracle_grid(w)
    prm = oracle_params(w, rtol)
    P, phi, rec = w.P0.copy(), None, []
    for s in range(steps):
        v = W.ramp_volts(amp, period, s)
        G.volt_hi = np.full((w.ny, w.nx), v)
        P, phi, st, _ = O.step(G, prm, P, phi, 1)
        assert st == O.OK
        rec.append([v, P[0].mean(), P[1].mean(), P[2].mean()])
    return P, phi, np.array(rec)


def run_batch(ws, steps, record_every=1, max_records=None):
    films = [Film(w) for w in ws]
    b = Batch(films, max_records=steps if max_records is None else max_records, record_every=record_every)
    for i, w in enumerate(ws):
        b.set_ramp(i, pf.PF_ZHI, *w.extra["ramp"])
    st, info = b.step(steps)
    loops = b.loops()
    out = [f.numpy() for f in films]
    infos = [b.film_info(i) for i in range(len(ws))]
    b.close()
    for f in films:
        f.close()
    return out, loops, info, infos


def test_fp64_batch_matches_oracle_with_ramps():
    ws = small_batch("fp64")
    out, loops, info, infos = run_batch(ws, 12)
    assert info["status"] == pf.PF_OK and info["graph_steps"] == 12
    assert loops.shape == (12, 3, 4)
    for i, w in enumerate(ws):
        Po, phio, rec = oracle_ramped(w, 12)
        P, phi = out[i]
        assert relerr(P, Po) <= FP64_TOL
        assert relerr(phi, phio) <= FP64_TOL
        assert np.abs(loops[:, i, 0] - rec[:, 0]).max() <= 1e-14 * max(1.0, np.abs(rec[:, 0]).max())
        assert np.abs(loops[:, i, 1:] - rec[:, 1:]).max() <= FP64_TOL * np.abs(P).max()
        assert infos[i]["total_iters"] > 0
    assert sum(i["total_iters"] for i in infos) == info["total_iters"]


def test_fp32_batch_equals_films_run_alone():
    """The batch graph runs the same kernels as a film stepped alone with the
    ramp voltage set from the host before every step: bitwise equal."""
    ws = [w.with_(rtol=1e-6) for w in small_batch("fp32", shapes=((32, 32, 16), (64, 32, 16)), n=4, seed=9)]
    out, loops, _, _ = run_batch(ws, 10)
    for i, w in enumerate(ws):
        f = Film(w)
        amp, period = w.extra["ramp"]
        for s in range(10):
            f.set_bc(pf.PF_ZHI, w.type_hi, np.full((w.ny, w.nx), W.ramp_volts(amp, period, s)))
            f.step(1)
        P, phi = f.numpy()
        f.close()
        assert np.array_equal(P, out[i][0]) and np.array_equal(phi, out[i][1])


def test_fp32_batch_vs_fp64_oracle():
    ws = [w.with_(rtol=1e-8) for w in small_batch("fp32", n=2, seed=11)]
    out, loops, _, _ = run_batch(ws, 12)
    for i, w in enumerate(ws):
        Po, _, rec = oracle_ramped(w, 12, rtol=1e-12)
        assert relerr(out[i][0], Po) <= FP32_TOL
        assert np.abs(loops[:, i, 3] - rec[:, 3]).max() <= FP32_TOL * np.abs(Po).max()


def test_record_every_and_capacity():
    ws = small_batch("fp64", n=2, seed=13)
    out, loops, _, _ = run_batch(ws, 10, record_every=3, max_records=2)
    assert loops.shape == (2, 2, 4)
    for i, w in enumerate(ws):
        amp, period = w.extra["ramp"]
        # record r is taken after batch step 3 (r + 1) - 1 with the voltage of that step
        assert loops[0, i, 0] == pytest.approx(W.ramp_volts(amp, period, 2), abs=1e-14)
        assert loops[1, i, 0] == pytest.approx(W.ramp_volts(amp, period, 5), abs=1e-14)


def test_batch_heun_and_refresh_match_films_alone():
    ws = [w.with_(rtol=1e-12) for w in small_batch("fp64", n=2, seed=17)]
    films = [Film(w, integrator=pf.PF_HEUN, poisson_every=2) for w in ws]
    b = Batch(films, max_records=5)
    b.step(5)
    got = [f.numpy() for f in films]
    b.close()
    for f in films:
        f.close()
    for i, w in enumerate(ws):
        f = Film(w, integrator=pf.PF_HEUN, poisson_every=2)
        f.step(5)
        ref = f.numpy()
        f.close()
        assert np.array_equal(got[i][0], ref[0]) and np.array_equal(got[i][1], ref[1])


def test_batch_argument_checks():
    ws = small_batch("fp64", n=2, seed=19)
    a = Film(ws[0])
    c = Film(ws[1], integrator=pf.PF_HEUN)
    with pytest.raises(pf.PfError) as e:
        Batch([a, c], max_records=1)
    assert e.value.status == pf.PF_ERR_ARG
    d = Film(ws[1])
    b = Batch([a, d], max_records=1)
    with pytest.raises(pf.PfError):
        b.set_ramp(2, pf.PF_ZHI, 1.0, 10.0)
    with pytest.raises(pf.PfError):
        b.set_ramp(0, pf.PF_ZHI, 1.0, -1.0)
    a.step(1)                      # a film stepped on its own leaves the batch out of step
    with pytest.raises(pf.PfError) as e:
        b.step(1)
    assert e.value.status == pf.PF_ERR_STATE
    b.close()
    for f in (a, c, d):
        f.close()


@pytest.mark.parametrize("vx,tz,bps", [(1, 1, 0), (1, 3, 1), (2, 8, 0), (2, 64, 2)])
def test_tilings_agree_fp64(vx, tz, bps):
    """Any valid tiling gives the default tiling's result up to the order of
    the reduction sums."""
    w = mixed_workload(40, 24, 12, 23, steps=6, rtol=1e-13)
    ref = Film(w)
    ref.step(6)
    Pr, phir = ref.numpy()
    ref.close()
    f = Film(w)
    pf.pf_set_tiling(f.ctx, vx, tz, bps)
    t = pf.pf_get_tiling(f.ctx)
    assert (t.vx, t.tz, t.blocks_per_sm) == (vx, min(tz, w.nz), bps)
    f.step(6)
    P, phi = f.numpy()
    f.close()
    assert relerr(P, Pr) <= 1e-12 and relerr(phi, phir) <= 1e-12


def test_tiling_rejects_bad_values():
    f = Film(mixed_workload(37, 24, 12, 3, steps=1))        # FP64, odd nx
    for bad in [(3, 4, 0), (4, 4, 0), (2, 4, 0), (1, 0, 0), (1, 65, 0), (1, 4, -1)]:
        with pytest.raises(pf.PfError) as e:
            pf.pf_set_tiling(f.ctx, *bad)
        assert e.value.status == pf.PF_ERR_ARG
    f.close()


def test_autotune_picks_a_candidate_and_results_hold():
    w = W.film_batch_hysteresis(nfilms=1, seed=4, steps=4, shapes=((64, 64, 32),))[0]
    res = AT.tune(w, steps=2, warmup=1)
    assert (res["vx"], res["tz"], res["blocks_per_sm"]) in [tuple(t) for t, _ in res["table"]]
    assert res["ms_per_iter"] <= res["default_ms_per_iter"]
    assert len(res["table"]) >= 6
    f = Film(w)
    AT.apply(f, res)
    f.set_bc(pf.PF_ZHI, w.type_hi, np.full((w.ny, w.nx), 1.0))
    f.step(4)
    P, _ = f.numpy()
    f.close()
    g = Film(w)
    g.set_bc(pf.PF_ZHI, w.type_hi, np.full((w.ny, w.nx), 1.0))
    g.step(4)
    P2, _ = g.numpy()
    g.close()
    assert relerr(P, P2) <= 1e-5
