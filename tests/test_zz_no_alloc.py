"""The allocation-free Poisson solve against the regular entry point.

pf_solve_potential_noalloc serves callers that cannot allocate device memory
(real-time loops that must not stall on the allocator, processes whose device
memory a fixed pool or another framework owns): it keeps its scratch in a
library-owned device array instead of a caller workspace.  Its result must
match pf_solve_potential on the same inputs, call after call (the array keeps
the previous call's contents, so the second call checks that nothing stale
leaks in), and the FP64 oracle.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_1202_6116_gb300 import build as B
from paper_1202_6116_gb300 import pf
from paper_1202_6116_gb300.film import Film, make_params

import oracle as O
from helpers import mixed_workload, oracle_grid, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pf.lib()


def regular_solve(w):
    f = Film(w)
    st, info = f.solve_potential()
    phi = f.phi.double().cpu().numpy()
    f.close()
    return phi, info


def noalloc_solve(w):
    dt = torch.float32 if w.precision == "fp32" else torch.float64
    P = torch.as_tensor(w.P0, dtype=dt, device="cuda").contiguous()
    phi = torch.zeros(w.shape, dtype=dt, device="cuda")
    stream = torch.cuda.current_stream()
    masks = [np.ascontiguousarray(a, dtype=t).reshape(-1) for a, t in
             ((w.type_lo, np.int8), (w.volt_lo, np.float64), (w.type_hi, np.int8), (w.volt_hi, np.float64))]
    st, info = pf.pf_solve_potential_noalloc(make_params(w), stream.cuda_stream, P, phi, *masks)
    return phi.double().cpu().numpy(), info.as_dict()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_noalloc_matches_regular_solve_twice(precision, tol):
    for seed in (31, 32):          # two calls in a row, different inputs
        w = mixed_workload(40, 24, 12, seed, precision=precision,
                           rtol=1e-12 if precision == "fp64" else 1e-7, amp=0.5)
        ref, rinfo = regular_solve(w)
        got, ginfo = noalloc_solve(w)
        assert relerr(got, ref) <= tol
        assert ginfo["last_iters"] == rinfo["last_iters"]


def test_noalloc_matches_oracle():
    w = mixed_workload(40, 24, 12, 34, precision="fp64", rtol=1e-13, amp=0.5)
    got, info = noalloc_solve(w)
    phio = O.solve_potential(oracle_grid(w), w.P0, rtol=1e-14)[0]
    assert relerr(got, phio) <= 1e-10
    assert info["last_iters"] > 0


def test_noalloc_rejects_oversized_grids():
    # 1M cells in FP64 need 32 MiB for the four Krylov vectors alone: just
    # beyond the array.  The buffers are full size, so that a failing size
    # check would give a wrong result here, never an out-of-bounds access.
    w = mixed_workload(128, 128, 64, 33)
    dt = torch.float64
    P = torch.zeros((3,) + w.shape, dtype=dt, device="cuda")
    phi = torch.zeros(w.shape, dtype=dt, device="cuda")
    with pytest.raises(pf.PfError) as e:
        pf.pf_solve_potential_noalloc(make_params(w), None, P, phi)
    assert e.value.status == pf.PF_ERR_ARG
    assert "scratch" in pf.pf_last_error(None)


def test_noalloc_rejects_host_pointers():
    w = mixed_workload(16, 8, 4, 35)
    P = torch.zeros((3,) + w.shape, dtype=torch.float64)          # host memory
    phi = torch.zeros(w.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(pf.PfError) as e:
        pf.pf_solve_potential_noalloc(make_params(w), None, P, phi)
    assert e.value.status == pf.PF_ERR_ARG
    assert "device" in pf.pf_last_error(None)


def test_noalloc_refuses_a_capturing_stream():
    """The call blocks, so it refuses to run while its stream is being
    captured (PF_ERR_STATE), before it enqueues anything."""
    w = mixed_workload(16, 8, 4, 36)
    P = torch.as_tensor(w.P0, dtype=torch.float64, device="cuda").contiguous()
    phi = torch.zeros(w.shape, dtype=torch.float64, device="cuda")
    x = torch.zeros(4, device="cuda")
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    status = {}
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            x.add_(1.0)
            status["st"], _ = pf.pf_solve_potential_noalloc(make_params(w), s.cuda_stream, P, phi,
                                                            ok=(pf.PF_OK, pf.PF_ERR_STATE))
    assert status["st"] == pf.PF_ERR_STATE
    assert "captur" in pf.pf_last_error(None)
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
