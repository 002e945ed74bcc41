"""CPU-side checks of the C ABI: the library builds, loads and exports every
function include/pf.h declares; parameter validation needs no GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_1202_6116_gb300 import build as B
from paper_1202_6116_gb300 import pf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pf.h")


@pytest.fixture(scope="module")
def L():
    B.build()
    return pf.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 10
    assert sorted(pf.EXPORTS) == names
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(r"\bT %s$" % n, out, flags=re.M), n


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pf.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(pf_params), sizeof(pf_step_info),'
                    ' offsetof(pf_params, poisson_rtol), offsetof(pf_step_info, last_relres),'
                    ' sizeof(pf_kernel_stat), offsetof(pf_kernel_stat, bytes), offsetof(pf_params, extrap_order));'
                    'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got == [C.sizeof(pf.pf_params), C.sizeof(pf.pf_step_info),
                   pf.pf_params.poisson_rtol.offset, pf.pf_step_info.last_relres.offset,
                   C.sizeof(pf.pf_kernel_stat), pf.pf_kernel_stat.bytes.offset, pf.pf_params.extrap_order.offset]


def good_params():
    p = pf.pf_params()
    p.nx, p.ny, p.nz, p.dx = 8, 6, 4, 1.0
    p.a1, p.a11, p.a12, p.g, p.L, p.dt = -1.0, 0.5, 0.8, 0.5, 1.0, 0.01
    p.poisson_rtol, p.poisson_maxit = 1e-10, 100
    return p


def test_workspace_bytes_and_validation(L):
    p = good_params()
    n = 8 * 6 * 4
    b64 = pf.pf_workspace_bytes(p)
    assert b64 >= 8 * (3 * n + 4 * n)
    p.precision = pf.PF_FP32
    b32 = pf.pf_workspace_bytes(p)
    assert 0 < b32 < b64
    for field, bad in (("nx", 0), ("nz", -3), ("dx", 0.0), ("precision", 7), ("solver", 9),
                       ("poisson_rtol", 0.0), ("poisson_maxit", 0), ("periodic_z", 2), ("dt", float("nan")),
                       ("integrator", 2), ("poisson_every", -1), ("n_air", 4), ("n_air", -1),
                       ("extrap_order", 4), ("extrap_order", -1)):
        q = good_params()
        setattr(q, field, bad)
        assert pf.pf_workspace_bytes(q) == 0, field
        ctx = C.c_void_p()
        assert L.pf_create(C.byref(q), None, C.byref(ctx)) == pf.PF_ERR_ARG, field
        assert ctx.value is None
        assert pf.pf_last_error(None) != ""
    q = good_params()
    q.reserved[1] = 1
    assert pf.pf_workspace_bytes(q) == 0
    q = good_params()
    q.n_air, q.periodic_z = 1, 1                   # air layers need non-periodic z
    assert pf.pf_workspace_bytes(q) == 0
    q.periodic_z = 0
    assert pf.pf_workspace_bytes(q) > 0
    q = good_params()
    q.flags = 16
    assert pf.pf_workspace_bytes(q) == 0
    q.flags = pf.PF_FLAG_WARM_LAST
    assert 0 < pf.pf_workspace_bytes(q) < pf.pf_workspace_bytes(good_params())   # no history fields
    q.flags = pf.PF_FLAG_NO_GRAPHS
    assert pf.pf_workspace_bytes(q) > 0


def test_null_context_calls_are_rejected(L):
    assert L.pf_step(None, 1, None) == pf.PF_ERR_ARG
    assert L.pf_set_bc(None, 0, None, None) == pf.PF_ERR_ARG
    assert L.pf_solve_potential(None, None) == pf.PF_ERR_ARG
    assert L.pf_bind(None, None, None, None, None, 0) == pf.PF_ERR_ARG
    assert L.pf_destroy(None) == pf.PF_OK


def test_workspace_of_the_extrapolated_start():
    """The extrapolated start costs three history fields (FP64); an FP32
    series adds the compensated remainder and the Krylov correction (five
    fields); the paper's last-potential start and the predictor-corrector
    need none."""
    p = good_params()
    p.nx, p.ny, p.nz = 32, 32, 32                 # fields of 128 or 256 KiB: no alignment padding
    n = 32 * 32 * 32
    for prec, word, fields in ((pf.PF_FP64, 8, 3), (pf.PF_FP32, 4, 5)):
        p.precision = prec
        p.flags, p.integrator = pf.PF_FLAG_PLAIN_FP32, pf.PF_EULER
        extrap = pf.pf_workspace_bytes(p)
        p.flags = pf.PF_FLAG_WARM_LAST | pf.PF_FLAG_PLAIN_FP32
        last = pf.pf_workspace_bytes(p)
        p.flags, p.integrator = pf.PF_FLAG_PLAIN_FP32, pf.PF_HEUN
        heun = pf.pf_workspace_bytes(p)
        assert extrap - last == fields * n * word
        assert heun == last
    p.integrator = pf.PF_EULER
    for order in (1, 2, 3):                       # the order changes no layout
        p.extrap_order = order
        assert pf.pf_workspace_bytes(p) == extrap


def test_workspace_of_the_compensated_state():
    """FP32 forward Euler keeps the polarization as P plus an FP32 remainder
    (3N bf16 values) unless PF_FLAG_PLAIN_FP32 is set; FP64, the
    predictor-corrector and adjoint contexts have none."""
    p = good_params()
    p.nx, p.ny, p.nz = 32, 32, 32
    n = 32 * 32 * 32
    p.precision = pf.PF_FP32
    comp = pf.pf_workspace_bytes(p)
    p.flags = pf.PF_FLAG_PLAIN_FP32
    plain = pf.pf_workspace_bytes(p)
    assert comp - plain == 3 * n * 2               # the remainder is stored in bf16
    p.flags = pf.PF_FLAG_ADJOINT
    adj = pf.pf_workspace_bytes(p)
    p.flags = pf.PF_FLAG_ADJOINT | pf.PF_FLAG_PLAIN_FP32
    assert adj == pf.pf_workspace_bytes(p)
    p.flags, p.integrator = 0, pf.PF_HEUN
    heun = pf.pf_workspace_bytes(p)
    p.flags = pf.PF_FLAG_PLAIN_FP32
    assert heun == pf.pf_workspace_bytes(p)
    p.integrator, p.flags, p.precision = pf.PF_EULER, 0, pf.PF_FP64
    b64 = pf.pf_workspace_bytes(p)
    p.flags = pf.PF_FLAG_PLAIN_FP32
    assert b64 == pf.pf_workspace_bytes(p)
