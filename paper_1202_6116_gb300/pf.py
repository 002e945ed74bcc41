"""Thin ctypes binding of the C ABI in ``include/pf.h`` (same names).

Argument marshalling only: every step of the computation runs in the CUDA
library ``_lib/libpfgb.so``.  There is no CPU fallback; if the library is
missing or cannot be loaded, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libpfgb.so")

PF_OK, PF_ERR_ARG, PF_ERR_CUDA, PF_ERR_NOCONV, PF_ERR_NONFINITE, PF_ERR_TIMEOUT, PF_ERR_STATE, \
    PF_ERR_NOTIMPL = range(8)
PF_FP64, PF_FP32 = 0, 1
PF_PCG_JACOBI, PF_PCG_MG = 0, 1
PF_ZLO, PF_ZHI = 0, 1
PF_NEUMANN, PF_DIRICHLET = 0, 1
PF_EULER, PF_HEUN = 0, 1
PF_FLAG_NO_GRAPHS = 1
PF_FLAG_ADJOINT = 2
PF_FLAG_WARM_LAST = 4
PF_FLAG_PLAIN_FP32 = 8

STATUS_NAMES = {0: "PF_OK", 1: "PF_ERR_ARG", 2: "PF_ERR_CUDA", 3: "PF_ERR_NOCONV", 4: "PF_ERR_NONFINITE",
                5: "PF_ERR_TIMEOUT", 6: "PF_ERR_STATE", 7: "PF_ERR_NOTIMPL"}

# Every symbol the header declares.
EXPORTS = ["pf_workspace_bytes", "pf_create", "pf_bind", "pf_set_bc", "pf_step", "pf_step_async", "pf_step_wait",
           "pf_step_host", "pf_true_residual",
           "pf_solve_potential", "pf_adjoint_step", "pf_diagnostics", "pf_profile_enable", "pf_profile_read", "pf_destroy",
           "pf_last_error", "pf_solve_potential_noalloc", "pf_set_noise", "pf_get_tiling", "pf_set_tiling",
           "pf_batch_workspace_bytes", "pf_batch_create", "pf_batch_set_ramp", "pf_batch_step",
           "pf_batch_film_info", "pf_batch_read_loops", "pf_batch_destroy", "pf_batch_last_error"]


class pf_params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("dx", C.c_double),
                ("a1", C.c_double), ("a11", C.c_double), ("a12", C.c_double),
                ("g", C.c_double), ("L", C.c_double), ("dt", C.c_double),
                ("precision", C.c_int32), ("solver", C.c_int32),
                ("poisson_rtol", C.c_double), ("poisson_maxit", C.c_int32),
                ("periodic_z", C.c_int32), ("has_eps", C.c_int32), ("flags", C.c_int32),
                ("integrator", C.c_int32), ("poisson_every", C.c_int32), ("n_air", C.c_int32),
                ("extrap_order", C.c_int32), ("reserved", C.c_int32 * 2)]


class pf_step_info(C.Structure):
    _fields_ = [("steps_done", C.c_int32), ("last_iters", C.c_int32), ("total_iters", C.c_int64),
                ("last_relres", C.c_double), ("nonconverged", C.c_int32), ("status", C.c_int32),
                ("kernel_launches", C.c_int64), ("graph_steps", C.c_int64),
                ("max_iters", C.c_int32), ("solves", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pf_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("idle_launches", C.c_int64),
                ("total_ms", C.c_double), ("bytes", C.c_double)]


class pf_tiling(C.Structure):
    _fields_ = [("vx", C.c_int32), ("tz", C.c_int32), ("blocks_per_sm", C.c_int32), ("mg_whole", C.c_int32)]


class PfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("GPU library %s not built: run paper_1202_6116_gb300.build.build() "
                               "(there is no CPU fallback)" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        vp, i32, sz = C.c_void_p, C.c_int32, C.c_size_t
        L.pf_workspace_bytes.restype = sz
        L.pf_workspace_bytes.argtypes = [C.POINTER(pf_params)]
        L.pf_create.restype = i32
        L.pf_create.argtypes = [C.POINTER(pf_params), vp, C.POINTER(vp)]
        L.pf_bind.restype = i32
        L.pf_bind.argtypes = [vp, vp, vp, vp, vp, sz]
        L.pf_set_bc.restype = i32
        L.pf_set_bc.argtypes = [vp, i32, vp, vp]
        L.pf_step.restype = i32
        L.pf_step.argtypes = [vp, i32, C.POINTER(pf_step_info)]
        L.pf_step_async.restype = i32
        L.pf_step_async.argtypes = [vp, i32]
        L.pf_step_wait.restype = i32
        L.pf_step_wait.argtypes = [vp, C.POINTER(pf_step_info)]
        L.pf_true_residual.restype = i32
        L.pf_true_residual.argtypes = [vp, vp, vp]
        L.pf_step_host.restype = i32
        L.pf_step_host.argtypes = [vp, vp, vp, i32, C.POINTER(pf_step_info)]
        L.pf_solve_potential.restype = i32
        L.pf_solve_potential.argtypes = [vp, C.POINTER(pf_step_info)]
        L.pf_diagnostics.restype = i32
        L.pf_diagnostics.argtypes = [vp, C.c_double, vp]
        L.pf_adjoint_step.restype = i32
        L.pf_adjoint_step.argtypes = [vp, vp, vp, vp, vp, vp]
        L.pf_profile_enable.restype = i32
        L.pf_profile_enable.argtypes = [vp, i32]
        L.pf_profile_read.restype = i32
        L.pf_profile_read.argtypes = [vp, vp, i32]
        L.pf_solve_potential_noalloc.restype = i32
        L.pf_solve_potential_noalloc.argtypes = [C.POINTER(pf_params), vp, vp, vp, vp, vp, vp, vp,
                                                 C.POINTER(pf_step_info)]
        L.pf_set_noise.restype = i32
        L.pf_set_noise.argtypes = [vp, C.c_double, C.c_uint64]
        L.pf_get_tiling.restype = i32
        L.pf_get_tiling.argtypes = [vp, C.POINTER(pf_tiling)]
        L.pf_set_tiling.restype = i32
        L.pf_set_tiling.argtypes = [vp, C.POINTER(pf_tiling)]
        L.pf_batch_workspace_bytes.restype = sz
        L.pf_batch_workspace_bytes.argtypes = [i32, C.c_int64]
        L.pf_batch_create.restype = i32
        L.pf_batch_create.argtypes = [vp, i32, vp, sz, C.c_int64, i32, C.POINTER(vp)]
        L.pf_batch_set_ramp.restype = i32
        L.pf_batch_set_ramp.argtypes = [vp, i32, i32, C.c_double, C.c_double]
        L.pf_batch_step.restype = i32
        L.pf_batch_step.argtypes = [vp, i32, C.POINTER(pf_step_info)]
        L.pf_batch_film_info.restype = i32
        L.pf_batch_film_info.argtypes = [vp, i32, C.POINTER(pf_step_info)]
        L.pf_batch_read_loops.restype = i32
        L.pf_batch_read_loops.argtypes = [vp, vp, C.c_int64, C.POINTER(C.c_int64)]
        L.pf_batch_destroy.restype = i32
        L.pf_batch_destroy.argtypes = [vp]
        L.pf_batch_last_error.restype = C.c_char_p
        L.pf_batch_last_error.argtypes = [vp]
        L.pf_destroy.restype = i32
        L.pf_destroy.argtypes = [vp]
        L.pf_last_error.restype = C.c_char_p
        L.pf_last_error.argtypes = [vp]
        _lib = L
    return _lib


def _addr(x):
    """Device/host address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError("cannot take the address of %r" % type(x))


def pf_last_error(ctx=None) -> str:
    return lib().pf_last_error(ctx).decode()


def check(status, ctx=None, ok=(PF_OK,)):
    if status not in ok:
        raise PfError(status, pf_last_error(ctx))
    return status


def pf_workspace_bytes(params: pf_params) -> int:
    return lib().pf_workspace_bytes(C.byref(params))


def pf_create(params: pf_params, stream=None):
    """Returns the opaque context handle (an int)."""
    ctx = C.c_void_p()
    st = lib().pf_create(C.byref(params), _addr(stream) if stream is not None else None, C.byref(ctx))
    check(st, None)
    return ctx.value


def pf_bind(ctx, P, phi, eps, workspace, workspace_bytes):
    return check(lib().pf_bind(ctx, _addr(P), _addr(phi), _addr(eps), _addr(workspace), workspace_bytes), ctx)


def pf_set_bc(ctx, face, type_xy, volts_xy=None):
    """type_xy: contiguous int8 host array (nx*ny); volts_xy: float64 host array or None."""
    return check(lib().pf_set_bc(ctx, face, _addr(type_xy), _addr(volts_xy)), ctx)


def pf_step(ctx, nsteps, ok=(PF_OK,)):
    info = pf_step_info()
    st = lib().pf_step(ctx, nsteps, C.byref(info))
    check(st, ctx, ok)
    return st, info


def pf_step_async(ctx, nsteps):
    """Enqueue nsteps steps; statistics stay on the device until pf_step_wait."""
    return check(lib().pf_step_async(ctx, int(nsteps)), ctx)


def pf_step_wait(ctx, ok=(PF_OK,)):
    info = pf_step_info()
    st = lib().pf_step_wait(ctx, C.byref(info))
    check(st, ctx, ok)
    return st, info


def pf_true_residual(ctx, P=None):
    """(||b(P) - A phi||_2, ||b(P)||_2, ||b(P) - A phi_c||_2) in FP64 for the
    bound phi and the compensated potential phi_c; P: a device tensor of the
    state (None: the bound P)."""
    out = (C.c_double * 3)()
    check(lib().pf_true_residual(ctx, _addr(P), C.cast(out, C.c_void_p)), ctx)
    return float(out[0]), float(out[1]), float(out[2])


def pf_step_host(ctx, P_host, phi_host, nsteps, ok=(PF_OK,)):
    info = pf_step_info()
    st = lib().pf_step_host(ctx, _addr(P_host), _addr(phi_host), nsteps, C.byref(info))
    check(st, ctx, ok)
    return st, info


def pf_solve_potential(ctx, ok=(PF_OK,)):
    info = pf_step_info()
    st = lib().pf_solve_potential(ctx, C.byref(info))
    check(st, ctx, ok)
    return st, info


def pf_adjoint_step(ctx, lam_in, lam_out, grad_params, grad_volts=None, ok=(PF_OK,)):
    """lam_in/lam_out: device 3N of the context precision; grad_params (4) and
    grad_volts (2*nx*ny or None): device float64, accumulated."""
    info = pf_step_info()
    st = lib().pf_adjoint_step(ctx, _addr(lam_in), _addr(lam_out), _addr(grad_params), _addr(grad_volts),
                               C.byref(info))
    check(st, ctx, ok)
    return st, info


DIAG_NAMES = ("mean_px", "mean_py", "mean_pz", "switched_fraction", "f_landau", "f_grad", "f_elec")


def pf_diagnostics(ctx, threshold=0.3):
    """Diagnostics of the bound state as a dict (names in DIAG_NAMES)."""
    out = (C.c_double * 7)()
    check(lib().pf_diagnostics(ctx, float(threshold), C.cast(out, C.c_void_p)), ctx)
    return dict(zip(DIAG_NAMES, list(out)))


def pf_profile_enable(ctx, enable=1):
    return check(lib().pf_profile_enable(ctx, int(enable)), ctx)


def pf_profile_read(ctx):
    """Per-kernel-family statistics as a list of dicts."""
    n = lib().pf_profile_read(ctx, None, 0)
    arr = (pf_kernel_stat * max(n, 1))()
    lib().pf_profile_read(ctx, C.cast(arr, C.c_void_p), n)
    return [dict(name=a.name.decode(), launches=a.launches, idle_launches=a.idle_launches,
                 total_ms=a.total_ms, bytes=a.bytes) for a in arr[:n]]


def pf_solve_potential_noalloc(params: pf_params, stream, P, phi, type_lo=None, volt_lo=None, type_hi=None,
                               volt_hi=None, ok=(PF_OK,)):
    """Poisson solve with no allocation (device P, phi; host int8 masks and
    float64 volts).  Returns (status, info)."""
    info = pf_step_info()
    st = lib().pf_solve_potential_noalloc(C.byref(params), _addr(stream), _addr(P), _addr(phi), _addr(type_lo),
                                          _addr(volt_lo), _addr(type_hi), _addr(volt_hi), C.byref(info))
    check(st, None, ok)
    return st, info


def pf_destroy(ctx):
    return lib().pf_destroy(ctx)


def pf_set_noise(ctx, sigma, seed=0):
    """Thermal random force: sigma sqrt(dt) standard normal draws per cell,
    component and step (sigma = 0: off)."""
    return check(lib().pf_set_noise(ctx, float(sigma), int(seed)), ctx)


def pf_get_tiling(ctx) -> pf_tiling:
    t = pf_tiling()
    check(lib().pf_get_tiling(ctx, C.byref(t)), ctx)
    return t


def pf_set_tiling(ctx, vx, tz, blocks_per_sm=0, mg_whole=0):
    t = pf_tiling(int(vx), int(tz), int(blocks_per_sm), int(mg_whole))
    return check(lib().pf_set_tiling(ctx, C.byref(t)), ctx)


def pf_batch_last_error(batch=None) -> str:
    return lib().pf_batch_last_error(batch).decode()


def _bcheck(status, batch=None, ok=(PF_OK,)):
    if status not in ok:
        raise PfError(status, pf_batch_last_error(batch))
    return status


def pf_batch_workspace_bytes(nfilms, max_records) -> int:
    return lib().pf_batch_workspace_bytes(int(nfilms), int(max_records))


def pf_batch_create(ctxs, workspace, workspace_bytes, max_records, record_every=1):
    """ctxs: list of context handles.  Returns the batch handle (an int)."""
    arr = (C.c_void_p * len(ctxs))(*ctxs)
    b = C.c_void_p()
    st = lib().pf_batch_create(C.cast(arr, C.c_void_p), len(ctxs), _addr(workspace), int(workspace_bytes),
                               int(max_records), int(record_every), C.byref(b))
    _bcheck(st, None)
    return b.value


def pf_batch_set_ramp(batch, film, face, amplitude, period):
    return _bcheck(lib().pf_batch_set_ramp(batch, int(film), int(face), float(amplitude), float(period)), batch)


def pf_batch_step(batch, nsteps, ok=(PF_OK,)):
    info = pf_step_info()
    st = lib().pf_batch_step(batch, int(nsteps), C.byref(info))
    _bcheck(st, batch, ok)
    return st, info


def pf_batch_film_info(batch, film):
    info = pf_step_info()
    _bcheck(lib().pf_batch_film_info(batch, int(film), C.byref(info)), batch)
    return info


def pf_batch_read_loops(batch, out, max_out):
    """out: float64 host array of at least max_out * nfilms * 4 entries.
    Returns the number of records stored on the device."""
    n = C.c_int64(0)
    _bcheck(lib().pf_batch_read_loops(batch, _addr(out), int(max_out), C.byref(n)), batch)
    return n.value


def pf_batch_destroy(batch):
    return lib().pf_batch_destroy(batch)
