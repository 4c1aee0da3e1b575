"""Python binding of libaf (include/af.h): one SSP-RK3 step of the
positivity-preserving Active Flux scheme for 2D ideal MHD with the
Godunov-Powell source term (arXiv:2506.04857), in FP64 on GB300 (sm_103a).

The functions mirror the C ABI one to one and only marshal arguments; every
step of the scheme runs in the CUDA kernels of libaf.  PyTorch provides device
memory (tensors) and streams.  There is no CPU fallback: if libaf cannot be
built or loaded, or no CUDA device is present, the calls raise.

A state is a list of four float64 arrays/tensors [8, nyp, nxp] (cell averages,
x-face, y-face and corner point values; af_sizes gives the extents).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "AF_BC_PERIODIC", "AF_BC_OUTFLOW", "AF_OK", "AFError", "af_create", "af_set_domain", "af_set_params",
    "af_get_params", "af_set_stream", "af_sizes", "af_set_state", "af_get_state", "af_get_stage", "af_rhs", "af_rhs_vjp", "af_adjoint_step",
    "af_adjoint_step_stages", "af_diagnostics", "af_sensor", "af_dt", "af_coeff_len", "af_record_coeffs",
    "af_freeze_coeffs", "af_stage_vjp", "af_adjoint_step_frozen", "AF_NCOEF",
    "af_stage",
    "af_step", "af_step_host", "af_sync", "af_status", "af_timing", "af_probe_fp64", "af_rhs_noalloc", "af_batch_create",
    "af_batch_set_domain", "af_batch_set_params", "af_batch_set_stream", "af_batch_set_state", "af_batch_get_state",
    "af_batch_step", "af_batch_graph", "af_batch_autotune", "af_batch_dt", "af_batch_status", "af_batch_last_error",
    "af_batch_destroy", "af_last_error", "af_destroy", "af_math_check", "Solver", "STAT_NAMES", "lib_path",
]

AF_BC_PERIODIC, AF_BC_OUTFLOW = 0, 1
AF_OK, AF_EINVAL, AF_ECUDA, AF_ENOMEM, AF_ENONPHYS, AF_EBOUNDS, AF_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
AF_NSTAT = 12
AF_ADJ_RECORDED = 1
AF_ADJ_DT = 2
AF_SIDE_OUTFLOW, AF_SIDE_REFLECTIVE, AF_SIDE_INFLOW = 0, 1, 2
AF_NCOEF = 13
# slots of a stage's coefficient block (af.h): theta^s and face theta of x- and y-faces, theta_ij,
# and the scaling-limiter theta*, theta** of the cell centres and of the three point classes
COEFF_SLOTS = ["ths_x", "ths_y", "th_x", "th_y", "th_src", "thc_1", "thc_2", "thp1_1", "thp1_2", "thp2_1",
               "thp2_2", "thp3_1", "thp3_2"]
STAT_NAMES = ["src_limited", "lambda_lt1", "face_theta_lt1", "sensor_lt099", "newton_solves", "newton_maxit",
              "shrink", "point_limited", "cfl_violations", "center_limited", "nonadmissible", "cell_shrink"]
_CODES = {AF_EINVAL: "AF_EINVAL", AF_ECUDA: "AF_ECUDA", AF_ENOMEM: "AF_ENOMEM", AF_ENONPHYS: "AF_ENONPHYS",
          AF_EBOUNDS: "AF_EBOUNDS", AF_ETIMEOUT: "AF_ETIMEOUT"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()


class AFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (_CODES.get(code, "AF_E?"), code, msg))
        self.code = code


class af_params(C.Structure):
    _fields_ = [("cfl", C.c_double), ("kappa", C.c_double), ("pp_on", C.c_int), ("src_cell_on", C.c_int),
                ("src_point_on", C.c_int), ("src_point_upwind", C.c_int)]


def lib_path() -> str:
    return os.path.join(_HERE, "_build", "libaf.so")


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            from . import build as _build
            path = _build.build()   # no-op when up to date; raises without nvcc
            lib = C.CDLL(path)
            vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
            pp = C.POINTER(C.c_void_p)
            lib.af_create.argtypes = [C.c_int, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_void_p)]
            lib.af_set_domain.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_double]
            lib.af_set_params.argtypes = [vp, C.POINTER(af_params)]
            lib.af_set_boundary.argtypes = [vp, ip, C.c_double, C.c_double, dp]
            lib.af_get_params.argtypes = [vp, C.POINTER(af_params)]
            lib.af_set_stream.argtypes = [vp, vp]
            lib.af_sizes.argtypes = [vp, C.c_int, ip, ip]
            lib.af_set_state.argtypes = [vp, pp, C.c_int]
            lib.af_get_state.argtypes = [vp, pp, C.c_int]
            lib.af_rhs.argtypes = [vp, pp, C.c_int]
            lib.af_dt.argtypes = [vp, vp, C.c_int]
            lib.af_sensor.argtypes = [vp, vp, vp, C.c_int]
            lib.af_stage.argtypes = [vp, C.c_int, vp, C.c_int]
            lib.af_step.argtypes = [vp, vp, C.c_int]
            lib.af_step_host.argtypes = [vp, pp, pp]
            lib.af_sync.argtypes = [vp]
            lib.af_get_stage.argtypes = [vp, pp, C.c_int]
            lib.af_rhs_vjp.argtypes = [vp, pp, pp, C.c_int]
            lib.af_divb.argtypes = [vp, vp, C.c_int]
            lib.af_diagnostics.argtypes = [vp, vp, C.c_int]
            lib.af_adjoint_step.argtypes = [vp, vp, C.c_int, pp, pp, C.c_int, C.c_int]
            lib.af_adjoint_step_stages.argtypes = [vp, vp, C.c_int, pp, pp, pp, pp, pp, C.c_int, C.c_int]
            lib.af_coeff_len.argtypes = [vp, C.POINTER(C.c_longlong)]
            lib.af_record_coeffs.argtypes = [vp, vp]
            lib.af_freeze_coeffs.argtypes = [vp, vp]
            lib.af_stage_vjp.argtypes = [vp, vp, C.c_int, vp, pp, pp, C.c_int]
            lib.af_adjoint_step_frozen.argtypes = [vp, vp, C.c_int, pp, pp, pp, vp, pp, pp, C.c_int, C.c_int]
            lib.af_status.argtypes = [vp, C.POINTER(C.c_longlong), C.c_int]
            lib.af_last_error.argtypes = [vp]
            lib.af_last_error.restype = C.c_char_p
            lib.af_destroy.argtypes = [vp]
            lib.af_destroy.restype = None
            lib.af_math_check.argtypes = [C.c_int, vp, vp, vp, C.c_longlong, vp]
            lib.af_timing.argtypes = [vp, C.c_int, vp, vp]
            lib.af_probe_fp64.argtypes = [vp, C.POINTER(C.c_double)]
            ip_ = C.POINTER(C.c_int)
            lib.af_batch_create.argtypes = [C.c_int, ip_, ip_, dp, ip_, C.POINTER(C.c_void_p)]
            lib.af_batch_set_domain.argtypes = [vp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
            lib.af_batch_set_params.argtypes = [vp, C.c_int, C.POINTER(af_params)]
            lib.af_batch_set_stream.argtypes = [vp, vp]
            lib.af_batch_set_state.argtypes = [vp, C.c_int, pp, C.c_int]
            lib.af_batch_get_state.argtypes = [vp, C.c_int, pp, C.c_int]
            lib.af_batch_step.argtypes = [vp, C.c_int]
            lib.af_batch_graph.argtypes = [vp, C.c_int]
            lib.af_batch_autotune.argtypes = [vp, C.c_int, ip_]
            lib.af_batch_dt.argtypes = [vp, C.c_int, dp]
            lib.af_batch_status.argtypes = [vp, C.POINTER(C.c_longlong), C.c_int]
            lib.af_batch_last_error.argtypes = [vp]
            lib.af_batch_last_error.restype = C.c_char_p
            lib.af_batch_destroy.argtypes = [vp]
            lib.af_batch_destroy.restype = None
            lib.af_rhs_noalloc.argtypes = [C.c_int, C.c_int, C.c_double, C.c_int, C.c_double, C.c_double,
                                           C.c_double, C.c_double, pp, pp, vp]
            lib.af1d_create.argtypes = [C.c_int, C.c_double, C.c_int, C.POINTER(C.c_void_p)]
            lib.af1d_set_domain.argtypes = [vp, C.c_double, C.c_double]
            lib.af1d_set_params.argtypes = [vp, C.POINTER(af_params)]
            lib.af1d_set_stream.argtypes = [vp, vp]
            lib.af1d_sizes.argtypes = [vp, C.c_int, ip]
            lib.af1d_set_state.argtypes = [vp, pp, C.c_int]
            lib.af1d_get_state.argtypes = [vp, pp, C.c_int]
            lib.af1d_get_stage.argtypes = [vp, pp, C.c_int]
            lib.af1d_dt.argtypes = [vp, vp, C.c_int]
            lib.af1d_stage.argtypes = [vp, C.c_int, vp, C.c_int]
            lib.af1d_step.argtypes = [vp, vp, C.c_int]
            lib.af1d_status.argtypes = [vp, C.POINTER(C.c_longlong), C.c_int]
            lib.af1d_timing.argtypes = [vp, C.c_int, vp, vp]
            lib.af1d_last_error.argtypes = [vp]
            lib.af1d_last_error.restype = C.c_char_p
            lib.af1d_destroy.argtypes = [vp]
            lib.af1d_destroy.restype = None
            _LIB = lib
        return _LIB


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise AFError(AF_ECUDA, "no CUDA device: libaf runs on the GPU only")
    return torch


def _check(ctx, rc: int):
    if rc != AF_OK:
        msg = af_last_error(ctx) if ctx else ""
        raise AFError(rc, msg)


def _ptr_array(ptrs: Sequence[int]):
    return (C.c_void_p * 4)(*ptrs)


def _is_tensor(x) -> bool:
    return type(x).__module__.startswith("torch")


# ---------------------------------------------------------------------------
# C ABI mirrors
# ---------------------------------------------------------------------------
def af_create(nx: int, ny: int, gamma: float, bc: int = AF_BC_PERIODIC):
    _torch()
    h = C.c_void_p()
    rc = _lib().af_create(int(nx), int(ny), float(gamma), int(bc), C.byref(h))
    if rc != AF_OK:
        raise AFError(rc, "af_create(%d, %d, %g, %d) failed" % (nx, ny, gamma, bc))
    return h


def af_set_domain(ctx, x0: float, x1: float, y0: float, y1: float) -> None:
    _check(ctx, _lib().af_set_domain(ctx, x0, x1, y0, y1))


def af_set_params(ctx, cfl: float = 0.2, kappa: float = 0.0, pp_on: bool = True, src_cell_on: bool = True,
                  src_point_on: bool = True, src_point_upwind: bool = False) -> None:
    p = af_params(cfl, kappa, int(pp_on), int(src_cell_on), int(src_point_on), int(src_point_upwind))
    _check(ctx, _lib().af_set_params(ctx, C.byref(p)))


def af_set_boundary(ctx, sides, inflow_lo: float = 0.0, inflow_hi: float = 0.0, inflow_U=None) -> None:
    """Per-side boundary kinds (left, right, bottom, top) of an outflow grid; see af.h."""
    sd = (C.c_int * 4)(*[int(v) for v in sides])
    u = (C.c_double * 8)(*([float(v) for v in inflow_U] if inflow_U is not None else [0.0] * 8))
    _check(ctx, _lib().af_set_boundary(ctx, sd, float(inflow_lo), float(inflow_hi), u))


def af_get_params(ctx) -> dict:
    p = af_params()
    _check(ctx, _lib().af_get_params(ctx, C.byref(p)))
    return {"cfl": p.cfl, "kappa": p.kappa, "pp_on": bool(p.pp_on), "src_cell_on": bool(p.src_cell_on),
            "src_point_on": bool(p.src_point_on), "src_point_upwind": bool(p.src_point_upwind)}


def af_set_stream(ctx, stream=None) -> None:
    """stream: a torch.cuda.Stream, a raw cudaStream_t (int) or None (legacy default stream)."""
    if stream is None:
        handle = None
    elif hasattr(stream, "cuda_stream"):
        handle = stream.cuda_stream
    else:
        handle = int(stream)
    _check(ctx, _lib().af_set_stream(ctx, handle))


def af_sizes(ctx, cls: int):
    a, b = C.c_int(), C.c_int()
    _check(ctx, _lib().af_sizes(ctx, cls, C.byref(a), C.byref(b)))
    return a.value, b.value


def _shapes(ctx):
    return [(8, af_sizes(ctx, c)[1], af_sizes(ctx, c)[0]) for c in range(4)]


def _marshal_in(ctx, U):
    """Pointers of a state given as CUDA tensors (on_device = 1) or host arrays (0)."""
    shapes = _shapes(ctx)
    if len(U) != 4:
        raise ValueError("a state has four DoF classes")
    if all(_is_tensor(u) and u.is_cuda for u in U):
        torch = _torch()
        keep = []
        for u, s in zip(U, shapes):
            if tuple(u.shape) != s or u.dtype != torch.float64:
                raise ValueError("class tensor must be float64 %s, got %s %s" % (s, u.dtype, tuple(u.shape)))
            keep.append(u.contiguous())
        return _ptr_array([k.data_ptr() for k in keep]), 1, keep
    keep = []
    for u, s in zip(U, shapes):
        a = u.detach().cpu().numpy() if _is_tensor(u) else np.asarray(u)
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != s:
            raise ValueError("class array must be %s, got %s" % (s, a.shape))
        keep.append(a)
    return _ptr_array([k.ctypes.data for k in keep]), 0, keep


def af_set_state(ctx, U) -> None:
    ptrs, dev, keep = _marshal_in(ctx, U)
    _check(ctx, _lib().af_set_state(ctx, ptrs, dev))
    del keep


def _outputs(ctx, out, device: bool):
    shapes = _shapes(ctx)
    if out is None:
        if device:
            torch = _torch()
            out = [torch.empty(s, dtype=torch.float64, device="cuda") for s in shapes]
        else:
            out = [np.empty(s) for s in shapes]
    on_dev = int(_is_tensor(out[0]) and out[0].is_cuda)
    ptrs = _ptr_array([o.data_ptr() if on_dev else o.ctypes.data for o in out])
    return out, ptrs, on_dev


def af_get_state(ctx, out=None, device: bool = True):
    out, ptrs, dev = _outputs(ctx, out, device)
    _check(ctx, _lib().af_get_state(ctx, ptrs, dev))
    return out


def _host_ptrs(ctx, U):
    """Pointers of host arrays that an asynchronous call keeps using after it returns: no
    conversion or copy is made (a temporary would be freed before the copy runs)."""
    shapes = _shapes(ctx)
    if len(U) != 4:
        raise ValueError("a state has four DoF classes")
    ptrs = []
    for u, s in zip(U, shapes):
        if _is_tensor(u):
            torch = _torch()
            if u.is_cuda or u.dtype != torch.float64 or not u.is_contiguous() or tuple(u.shape) != s:
                raise ValueError("host tensor must be a contiguous CPU float64 %s" % (s,))
            ptrs.append(u.data_ptr())
        elif isinstance(u, np.ndarray):
            if u.dtype != np.float64 or not u.flags.c_contiguous or u.shape != s:
                raise ValueError("host array must be a C-contiguous float64 %s" % (s,))
            ptrs.append(u.ctypes.data)
        else:
            raise ValueError("af_step_host takes numpy arrays or CPU tensors")
    return _ptr_array(ptrs)


def af_step_host(ctx, U_in, U_out) -> None:
    """One step of a host-resident state, pipelined (see af.h): U_in and U_out are four
    host arrays (pinned for overlap) that must stay alive and untouched until af_sync."""
    _check(ctx, _lib().af_step_host(ctx, _host_ptrs(ctx, U_in), _host_ptrs(ctx, U_out)))


def af_sync(ctx) -> None:
    _check(ctx, _lib().af_sync(ctx))


def af_get_stage(ctx, out=None, device: bool = True):
    """The result of the most recent stage (U1, U2 or U^{n+1})."""
    out, ptrs, dev = _outputs(ctx, out, device)
    _check(ctx, _lib().af_get_stage(ctx, ptrs, dev))
    return out


def af_diagnostics(ctx, out=None):
    """Run diagnostics of the current state: {"min_rho": [4 classes], "min_p": [4 classes],
    "mass": dx dy sum of the cell-average densities}.  With out (a 9-element CUDA float64
    tensor) the raw values are written on the device without synchronising."""
    if out is not None:
        _check(ctx, _lib().af_diagnostics(ctx, out.data_ptr(), 1))
        return out
    res = (C.c_double * 9)()
    _check(ctx, _lib().af_diagnostics(ctx, C.cast(res, C.c_void_p), 0))
    v = [float(x) for x in res]
    return {"min_rho": v[0:4], "min_p": v[4:8], "mass": v[8]}


def af_divb(ctx, out=None):
    """(divB_1, divB_2) of the current state (Example 4.4); with out (a 2-element CUDA float64
    tensor) the values are written on the device without synchronising."""
    if out is not None:
        _check(ctx, _lib().af_divb(ctx, out.data_ptr(), 1))
        return out
    res = (C.c_double * 2)()
    _check(ctx, _lib().af_divb(ctx, C.cast(res, C.c_void_p), 0))
    return float(res[0]), float(res[1])


def af_rhs_vjp(ctx, v, out=None, device: bool = True):
    """(dL/dU)^T v at the current state (v: four arrays/tensors in the state layout)."""
    ptrs, dev, keep = _marshal_in(ctx, v)
    out, optrs, odev = _outputs(ctx, out, device)
    if dev != odev:
        raise ValueError("v and out must both be on the device or both on the host")
    _check(ctx, _lib().af_rhs_vjp(ctx, ptrs, optrs, dev))
    del keep
    return out


def af_adjoint_step(ctx, dt, lam, out=None, device: bool = True, recorded: bool = False,
                    dt_sensitivity: bool = False):
    """lambda^n = (dU^{n+1}/dU^n)^T lambda^{n+1} for one step from the current state with time step dt
    (a float or a one-element CUDA float64 tensor).  recorded=True (AF_ADJ_RECORDED): the caller has
    checked, from the forward step's counters, that no limiter acted in its last stage.
    dt_sensitivity=True (AF_ADJ_DT): dt is differentiated as the function of U^n that af_step forms."""
    ptrs, dev, keep = _marshal_in(ctx, lam)
    out, optrs, odev = _outputs(ctx, out, device)
    if dev != odev:
        raise ValueError("lam and out must both be on the device or both on the host")
    flags = (AF_ADJ_RECORDED if recorded else 0) | (AF_ADJ_DT if dt_sensitivity else 0)
    if _is_tensor(dt) and dt.is_cuda:
        rc = _lib().af_adjoint_step(ctx, dt.data_ptr(), 1, ptrs, optrs, dev, flags)
    else:
        v = C.c_double(float(dt))
        rc = _lib().af_adjoint_step(ctx, C.cast(C.byref(v), C.c_void_p), 0, ptrs, optrs, dev, flags)
    _check(ctx, rc)
    del keep
    return out


def af_adjoint_step_stages(ctx, dt, U1, U2, lam, U3=None, out=None, device: bool = True,
                           dt_sensitivity: bool = False):
    """af_adjoint_step with the forward step's stage states U1, U2 (and U3 = U^{n+1} for
    dt_sensitivity) given, as af_get_stage returned them, instead of recomputed.  The caller
    has checked, from the forward step's counters, that no positivity limiter acted."""
    ptrs, dev, keep = _marshal_in(ctx, lam)
    p1, d1, k1 = _marshal_in(ctx, U1)
    p2, d2, k2 = _marshal_in(ctx, U2)
    if U3 is not None:
        p3, d3, k3 = _marshal_in(ctx, U3)
    else:
        p3, d3, k3 = None, dev, None
    out, optrs, odev = _outputs(ctx, out, device)
    if len({dev, odev, d1, d2, d3}) != 1:
        raise ValueError("lam, out and the stage states must all be on the device or all on the host")
    flags = AF_ADJ_DT if dt_sensitivity else 0
    if _is_tensor(dt) and dt.is_cuda:
        dtp, dtd = dt.data_ptr(), 1
    else:
        v = C.c_double(float(dt))
        dtp, dtd = C.cast(C.byref(v), C.c_void_p), 0
    _check(ctx, _lib().af_adjoint_step_stages(ctx, dtp, dtd, p1, p2, p3, ptrs, optrs, dev, flags))
    del keep, k1, k2, k3
    return out


def _dt_arg(dt):
    if _is_tensor(dt) and dt.is_cuda:
        return dt.data_ptr(), 1, None
    v = C.c_double(float(dt))
    return C.cast(C.byref(v), C.c_void_p), 0, v


def af_coeff_len(ctx) -> int:
    """Doubles in one stage's block of limiter coefficients (AF_NCOEF index grids)."""
    n = C.c_longlong()
    _check(ctx, _lib().af_coeff_len(ctx, C.byref(n)))
    return n.value


def _coeff_ptr(ctx, buf, blocks: int):
    torch = _torch()
    if buf is None:
        return None
    if not (_is_tensor(buf) and buf.is_cuda) or buf.dtype != torch.float64 or not buf.is_contiguous():
        raise ValueError("coefficients: a contiguous CUDA float64 tensor")
    if buf.numel() < blocks * af_coeff_len(ctx):
        raise ValueError("coefficients: need %d doubles" % (blocks * af_coeff_len(ctx)))
    return buf.data_ptr()


def af_record_coeffs(ctx, buf) -> None:
    """buf: a CUDA float64 tensor of 3 * af_coeff_len(ctx) doubles, or None to stop recording."""
    _check(ctx, _lib().af_record_coeffs(ctx, _coeff_ptr(ctx, buf, 3)))


def af_freeze_coeffs(ctx, buf) -> None:
    """buf: recorded coefficients (3 stage blocks), or None to return to the limiters."""
    _check(ctx, _lib().af_freeze_coeffs(ctx, _coeff_ptr(ctx, buf, 3)))


def af_stage_vjp(ctx, dt, coeffs, lam, out=None, device: bool = True):
    """(d FE(U)/dU)^T lam of the forward-Euler stage of the current state along the branch
    frozen at coeffs (one stage block, CUDA float64 tensor)."""
    ptrs, dev, keep = _marshal_in(ctx, lam)
    out, optrs, odev = _outputs(ctx, out, device)
    if dev != odev:
        raise ValueError("lam and out must both be on the device or both on the host")
    dtp, dtd, dtk = _dt_arg(dt)
    _check(ctx, _lib().af_stage_vjp(ctx, dtp, dtd, _coeff_ptr(ctx, coeffs, 1), ptrs, optrs, dev))
    del keep, dtk
    return out


def af_adjoint_step_frozen(ctx, dt, U1, U2, coeffs, lam, U3=None, out=None, device: bool = True,
                           dt_sensitivity: bool = False):
    """The adjoint of one step along its recorded branch (af.h): U1, U2 (and U3) the forward
    step's stage states, coeffs its recorded coefficients (3 blocks)."""
    ptrs, dev, keep = _marshal_in(ctx, lam)
    p1, d1, k1 = _marshal_in(ctx, U1)
    p2, d2, k2 = _marshal_in(ctx, U2)
    if U3 is not None:
        p3, d3, k3 = _marshal_in(ctx, U3)
    else:
        p3, d3, k3 = None, dev, None
    out, optrs, odev = _outputs(ctx, out, device)
    if len({dev, odev, d1, d2, d3}) != 1:
        raise ValueError("lam, out and the stage states must all be on the device or all on the host")
    dtp, dtd, dtk = _dt_arg(dt)
    flags = AF_ADJ_DT if dt_sensitivity else 0
    _check(ctx, _lib().af_adjoint_step_frozen(ctx, dtp, dtd, p1, p2, p3, _coeff_ptr(ctx, coeffs, 3), ptrs, optrs,
                                              dev, flags))
    del keep, k1, k2, k3, dtk
    return out


def af_rhs(ctx, out=None, device: bool = True):
    out, ptrs, dev = _outputs(ctx, out, device)
    _check(ctx, _lib().af_rhs(ctx, ptrs, dev))
    return out


def af_sensor(ctx, device: bool = True):
    """theta^s at the x-faces [ny, nxf] and y-faces [nyf, nx] of the current state."""
    (nxf, ny), (nx, nyf) = af_sizes(ctx, 1), af_sizes(ctx, 2)
    if device:
        torch = _torch()
        tx = torch.empty((ny, nxf), dtype=torch.float64, device="cuda")
        ty = torch.empty((nyf, nx), dtype=torch.float64, device="cuda")
        _check(ctx, _lib().af_sensor(ctx, tx.data_ptr(), ty.data_ptr(), 1))
    else:
        tx, ty = np.empty((ny, nxf)), np.empty((nyf, nx))
        _check(ctx, _lib().af_sensor(ctx, tx.ctypes.data, ty.ctypes.data, 0))
    return tx, ty


def af_dt(ctx, out=None) -> Optional[float]:
    """dt of the current state.  out: None (returns a float, synchronises) or a
    one-element CUDA float64 tensor that receives dt in stream order."""
    if out is None:
        v = C.c_double()
        _check(ctx, _lib().af_dt(ctx, C.cast(C.byref(v), C.c_void_p), 0))
        return v.value
    _check(ctx, _lib().af_dt(ctx, out.data_ptr(), 1))
    return None


def af_stage(ctx, s: int, dt=None) -> None:
    """dt: None (value from the last af_dt/af_step), a float, or a CUDA float64 tensor."""
    if dt is None:
        _check(ctx, _lib().af_stage(ctx, s, None, 0))
    elif _is_tensor(dt) and dt.is_cuda:
        _check(ctx, _lib().af_stage(ctx, s, dt.data_ptr(), 1))
    else:
        v = C.c_double(float(dt))
        _check(ctx, _lib().af_stage(ctx, s, C.cast(C.byref(v), C.c_void_p), 0))


def af_step(ctx, dt_out=None) -> Optional[float]:
    """One SSP-RK3 step.  dt_out: None (returns dt as a float, synchronises),
    False (returns nothing, no synchronisation) or a CUDA float64 tensor."""
    if dt_out is False:
        _check(ctx, _lib().af_step(ctx, None, 0))
        return None
    if dt_out is None:
        v = C.c_double()
        _check(ctx, _lib().af_step(ctx, C.cast(C.byref(v), C.c_void_p), 0))
        return v.value
    _check(ctx, _lib().af_step(ctx, dt_out.data_ptr(), 1))
    return None


def af_status(ctx, reset: bool = False):
    """(return code, counters as a dict) after synchronising the stream."""
    cnt = (C.c_longlong * AF_NSTAT)()
    rc = _lib().af_status(ctx, cnt, int(reset))
    return rc, dict(zip(STAT_NAMES, [int(v) for v in cnt]))


KERNEL_NAMES = ["k_pointdata", "k_dt", "k_points", "k_faces", "k_cells", "k_final", "k_repair", "k_points_slow",
                "k_cells_slow"]


def af_timing(ctx, enable: bool):
    """enable=True starts per-kernel event timing; enable=False stops it and
    returns {kernel: (total ms, launches)}."""
    if enable:
        _check(ctx, _lib().af_timing(ctx, 1, None, None))
        return None
    ms = (C.c_double * len(KERNEL_NAMES))()
    n = (C.c_longlong * len(KERNEL_NAMES))()
    _check(ctx, _lib().af_timing(ctx, 0, C.cast(ms, C.c_void_p), C.cast(n, C.c_void_p)))
    return {k: (ms[i], int(n[i])) for i, k in enumerate(KERNEL_NAMES)}


def af_probe_fp64(stream=None) -> float:
    """Measured FP64 FMA throughput of the current device in TFLOP/s."""
    handle = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    v = C.c_double()
    rc = _lib().af_probe_fp64(handle, C.byref(v))
    if rc != AF_OK:
        raise AFError(rc, "af_probe_fp64 failed")
    return v.value


AF_NOALLOC_MAX_POINTS = 4225


def _noalloc_check(nx: int, ny: int, bc: int, U, out) -> None:
    """The C entry point cannot see extents: every class tensor must be a contiguous CUDA float64
    tensor on the current device with the [8][ey][ex] layout of the grid, and no output may
    overlap an input (the kernels read U while they write dUdt)."""
    torch = _torch()
    if len(U) != 4 or len(out) != 4:
        raise ValueError("U and out each hold four DoF classes")
    if nx < 4 or ny < 4 or bc not in (AF_BC_PERIODIC, AF_BC_OUTFLOW):
        raise ValueError("af_rhs_noalloc: need nx, ny >= 4 and a periodic or outflow grid")
    ex = [nx, nx + (bc == AF_BC_OUTFLOW), nx, nx + (bc == AF_BC_OUTFLOW)]
    ey = [ny, ny, ny + (bc == AF_BC_OUTFLOW), ny + (bc == AF_BC_OUTFLOW)]
    dev = torch.cuda.current_device()
    spans = []
    for name, group in (("U", U), ("out", out)):
        for c, t in enumerate(group):
            if not (_is_tensor(t) and t.is_cuda) or t.dtype != torch.float64 or not t.is_contiguous():
                raise ValueError("%s[%d] must be a contiguous CUDA float64 tensor" % (name, c))
            if t.device.index != dev:
                raise ValueError("%s[%d] is on cuda:%s, the current device is cuda:%d" % (name, c, t.device.index, dev))
            if tuple(t.shape) != (8, ey[c], ex[c]):
                raise ValueError("%s[%d] must have shape %s, got %s" % (name, c, (8, ey[c], ex[c]), tuple(t.shape)))
            spans.append((name, t.data_ptr(), t.data_ptr() + t.numel() * 8))
    for n1, a0, a1 in spans[4:]:
        for n0, b0, b1 in spans:
            if n0 == "U" and a0 < b1 and b0 < a1:
                raise ValueError("an output of af_rhs_noalloc overlaps an input")


def af_rhs_noalloc(nx: int, ny: int, gamma: float, bc: int, domain, U, out, stream=None) -> None:
    """af_rhs computed in the library's static scratch, with no device allocation.

    For callers that cannot allocate device memory on their hot path.  U and
    out are lists of four CUDA float64 tensors in the state layout; grids with
    (nx [+1 outflow]) x (ny [+1 outflow]) > AF_NOALLOC_MAX_POINTS are rejected
    (AF_EBOUNDS).  Calls share one scratch array: do not overlap them on the GPU."""
    handle = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _noalloc_check(int(nx), int(ny), int(bc), U, out)
    ins = _ptr_array([u.data_ptr() for u in U])
    outs = _ptr_array([o.data_ptr() for o in out])
    rc = _lib().af_rhs_noalloc(int(nx), int(ny), float(gamma), int(bc), *[float(v) for v in domain], ins, outs,
                               handle)
    if rc != AF_OK:
        raise AFError(rc, "af_rhs_noalloc(%d, %d) failed" % (nx, ny))


def af_last_error(ctx) -> str:
    r = _lib().af_last_error(ctx)
    return r.decode() if r else ""


def af_destroy(ctx) -> None:
    if ctx:
        _lib().af_destroy(ctx)


# values of x per result and of y (per result, or in all) that each af_math_check op reads
_MATH_X_PER = {9: 8, 10: 40}
_MATH_Y = {1: "n", 3: "n", 4: "n", 5: "n", 6: "n", 7: "n", 9: 1, 10: 3}


def af_math_check(op: int, x, y, out, stream=None) -> None:
    """n = out.numel() results of the FP64 helpers or certificates (see af.h); every
    buffer is checked here, since the C entry point cannot see their extents."""
    import torch
    if op not in range(11):
        raise ValueError("af_math_check: op %d outside 0..10" % op)
    n = out.numel()
    need = {"x": (x, n * _MATH_X_PER.get(op, 1)), "out": (out, n)}
    ny = _MATH_Y.get(op)
    if ny is not None:
        if y is None:
            raise ValueError("af_math_check: op %d reads y" % op)
        need["y"] = (y, n if ny == "n" else ny)
    for name, (t, size) in need.items():
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.device == out.device):
            raise ValueError("af_math_check: %s must be a contiguous CUDA float64 tensor on out's device" % name)
        if t.numel() < size:
            raise ValueError("af_math_check: %s holds %d values, op %d reads %d" % (name, t.numel(), op, size))
    handle = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    rc = _lib().af_math_check(op, x.data_ptr(), None if ny is None else y.data_ptr(), out.data_ptr(), n, handle)
    if rc != AF_OK:
        raise AFError(rc, "af_math_check failed")


# ---------------------------------------------------------------------------
# batched ensembles
# ---------------------------------------------------------------------------
def _bcheck(b, rc: int):
    if rc != AF_OK:
        r = _lib().af_batch_last_error(b)
        raise AFError(rc, r.decode() if r else "")


def af_batch_create(nx, ny, gamma, bc):
    """nx, ny, gamma, bc: per-run sequences of equal length."""
    _torch()
    n = len(nx)
    a = (C.c_int * n)(*[int(v) for v in nx])
    b_ = (C.c_int * n)(*[int(v) for v in ny])
    g = (C.c_double * n)(*[float(v) for v in gamma])
    c = (C.c_int * n)(*[int(v) for v in bc])
    h = C.c_void_p()
    rc = _lib().af_batch_create(n, a, b_, g, c, C.byref(h))
    if rc != AF_OK:
        raise AFError(rc, "af_batch_create(%d runs) failed" % n)
    return h


def af_batch_set_domain(b, run, x0, x1, y0, y1):
    _bcheck(b, _lib().af_batch_set_domain(b, run, x0, x1, y0, y1))


def af_batch_set_params(b, run, cfl=0.2, kappa=0.0, pp_on=True, src_cell_on=True, src_point_on=True,
                        src_point_upwind=False):
    p = af_params(cfl, kappa, int(pp_on), int(src_cell_on), int(src_point_on), int(src_point_upwind))
    _bcheck(b, _lib().af_batch_set_params(b, run, C.byref(p)))


def af_batch_set_stream(b, stream=None):
    handle = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _bcheck(b, _lib().af_batch_set_stream(b, handle))


def af_batch_set_state(b, run, U):
    dev = all(_is_tensor(u) and u.is_cuda for u in U)
    keep = [u.contiguous() if dev else np.ascontiguousarray(u.detach().cpu().numpy() if _is_tensor(u) else u,
                                                             dtype=np.float64) for u in U]
    ptrs = _ptr_array([k.data_ptr() if dev else k.ctypes.data for k in keep])
    _bcheck(b, _lib().af_batch_set_state(b, run, ptrs, int(dev)))


def af_batch_get_state(b, run, out):
    """out: four arrays/tensors of the run's class shapes (CUDA tensors or numpy)."""
    dev = int(_is_tensor(out[0]) and out[0].is_cuda)
    ptrs = _ptr_array([o.data_ptr() if dev else o.ctypes.data for o in out])
    _bcheck(b, _lib().af_batch_get_state(b, run, ptrs, dev))
    return out


def af_batch_step(b, nsteps: int = 1):
    _bcheck(b, _lib().af_batch_step(b, int(nsteps)))


def af_batch_graph(b, enable: bool = True):
    _bcheck(b, _lib().af_batch_graph(b, int(enable)))


def af_batch_autotune(b, reps: int = 3):
    ch = (C.c_int * 4)()
    _bcheck(b, _lib().af_batch_autotune(b, int(reps), ch))
    return {"tile": (ch[0], ch[1]), "blocks_per_sm_cap": ch[2], "us_per_stage": ch[3]}


def af_batch_dt(b, run: int) -> float:
    v = C.c_double()
    _bcheck(b, _lib().af_batch_dt(b, run, C.byref(v)))
    return v.value


def af_batch_status(b, reset: bool = False):
    cnt = (C.c_longlong * AF_NSTAT)()
    rc = _lib().af_batch_status(b, cnt, int(reset))
    return rc, dict(zip(STAT_NAMES, [int(v) for v in cnt]))


def af_batch_last_error(b) -> str:
    r = _lib().af_batch_last_error(b)
    return r.decode() if r else ""


def af_batch_destroy(b):
    if b:
        _lib().af_batch_destroy(b)


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
class Solver:
    """Owns one libaf context.  Example:

        s = Solver(512, 512, 5/3, AF_BC_PERIODIC, domain=(0, 2*pi, 0, 2*pi), kappa=1.0)
        s.set_state(U0)          # four float64 arrays/tensors
        dt = s.step()
        U = s.get_state()        # CUDA tensors
    """

    def __init__(self, nx: int, ny: int, gamma: float, bc: int = AF_BC_PERIODIC, domain=(0.0, 1.0, 0.0, 1.0),
                 cfl: float = 0.2, kappa: float = 0.0, pp_on: bool = True, src_cell_on: bool = True,
                 src_point_on: bool = True, stream=None, sides=None, inflow=None, src_point_upwind: bool = False):
        """sides: per-side boundary kinds (left, right, bottom, top) of an outflow grid;
        inflow: (lo, hi, conserved state) for AF_SIDE_INFLOW sides."""
        self.ctx = af_create(nx, ny, gamma, bc)
        self.nx, self.ny, self.bc = nx, ny, bc
        af_set_domain(self.ctx, *domain)
        af_set_params(self.ctx, cfl, kappa, pp_on, src_cell_on, src_point_on, src_point_upwind)
        if stream is not None:
            af_set_stream(self.ctx, stream)
        if sides is not None and any(sides):
            lo, hi, U = inflow if inflow is not None else (0.0, 0.0, None)
            af_set_boundary(self.ctx, sides, lo, hi, U)

    def sizes(self):
        return [af_sizes(self.ctx, c) for c in range(4)]

    def set_state(self, U):
        af_set_state(self.ctx, U)

    def get_state(self, out=None, device: bool = True):
        return af_get_state(self.ctx, out, device)

    def get_stage(self, out=None, device: bool = True):
        return af_get_stage(self.ctx, out, device)

    def rhs(self, out=None, device: bool = True):
        return af_rhs(self.ctx, out, device)

    def dt(self, out=None):
        return af_dt(self.ctx, out)

    def divb(self, out=None):
        return af_divb(self.ctx, out)

    def diagnostics(self, out=None):
        return af_diagnostics(self.ctx, out)

    def sensor(self, device: bool = True):
        return af_sensor(self.ctx, device)

    def stage(self, s: int, dt=None):
        af_stage(self.ctx, s, dt)

    def step(self, dt_out=None):
        return af_step(self.ctx, dt_out)

    def step_host(self, U_in, U_out):
        af_step_host(self.ctx, U_in, U_out)

    def sync(self):
        af_sync(self.ctx)

    def status(self, reset: bool = False):
        return af_status(self.ctx, reset)

    def timing(self, enable: bool):
        return af_timing(self.ctx, enable)

    def close(self):
        if self.ctx:
            af_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# The 1D scheme (af1d_*): states are [averages [8, n], point values [8, nf]]
# ---------------------------------------------------------------------------
def _check1d(ctx, rc: int):
    if rc != AF_OK:
        raise AFError(rc, _lib().af1d_last_error(ctx).decode() if ctx else "")


def af1d_create(n: int, gamma: float, bc: int = AF_BC_PERIODIC):
    h = C.c_void_p()
    rc = _lib().af1d_create(n, gamma, bc, C.byref(h))
    if rc != AF_OK:
        raise AFError(rc, "af1d_create failed")
    return h


def af1d_sizes(ctx):
    a, b = C.c_int(), C.c_int()
    _check1d(ctx, _lib().af1d_sizes(ctx, 0, C.byref(a)))
    _check1d(ctx, _lib().af1d_sizes(ctx, 1, C.byref(b)))
    return a.value, b.value


def _marshal1d(ctx, U, out: bool = False, device: bool = True):
    n, nf = af1d_sizes(ctx)
    shapes = [(8, n), (8, nf)]
    if U is None:
        if device:
            torch = _torch()
            U = [torch.empty(s, dtype=torch.float64, device="cuda") for s in shapes]
        else:
            U = [np.empty(s) for s in shapes]
    keep = []
    ptrs = []
    on_dev = int(_is_tensor(U[0]) and U[0].is_cuda)
    for u, s in zip(U, shapes):
        if on_dev:
            if tuple(u.shape) != s or not u.is_contiguous():
                raise ValueError("1D array must be a contiguous %s tensor" % (s,))
            ptrs.append(u.data_ptr())
        else:
            a = u if out else np.ascontiguousarray(u, dtype=np.float64)
            if a.shape != s:
                raise ValueError("1D array must be %s, got %s" % (s, a.shape))
            keep.append(a)
            ptrs.append(a.ctypes.data)
    return U, _ptr_array(ptrs), on_dev, keep


def af1d_set_domain(ctx, x0: float, x1: float) -> None:
    _check1d(ctx, _lib().af1d_set_domain(ctx, float(x0), float(x1)))


def af1d_set_stream(ctx, stream=None) -> None:
    _check1d(ctx, _lib().af1d_set_stream(ctx, C.c_void_p(stream.cuda_stream if stream is not None else 0)))


def af1d_set_params(ctx, cfl: float = 0.2, kappa: float = 0.0, pp_on: bool = True) -> None:
    p = af_params(cfl, kappa, int(pp_on), 0, 0)
    _check1d(ctx, _lib().af1d_set_params(ctx, C.byref(p)))


def af1d_set_state(ctx, U) -> None:
    _, ptrs, dev, keep = _marshal1d(ctx, U)
    _check1d(ctx, _lib().af1d_set_state(ctx, ptrs, dev))
    del keep


def af1d_get_state(ctx, out=None, device: bool = True):
    out, ptrs, dev, keep = _marshal1d(ctx, out, out=True, device=device)
    _check1d(ctx, _lib().af1d_get_state(ctx, ptrs, dev))
    return out


def af1d_get_stage(ctx, out=None, device: bool = True):
    out, ptrs, dev, keep = _marshal1d(ctx, out, out=True, device=device)
    _check1d(ctx, _lib().af1d_get_stage(ctx, ptrs, dev))
    return out


def af1d_dt(ctx) -> float:
    d = C.c_double()
    _check1d(ctx, _lib().af1d_dt(ctx, C.cast(C.byref(d), C.c_void_p), 0))
    return d.value


def af1d_stage(ctx, s: int, dt=None) -> None:
    if dt is None:
        rc = _lib().af1d_stage(ctx, s, None, 0)
    elif _is_tensor(dt) and dt.is_cuda:
        rc = _lib().af1d_stage(ctx, s, dt.data_ptr(), 1)
    else:
        v = C.c_double(float(dt))
        rc = _lib().af1d_stage(ctx, s, C.cast(C.byref(v), C.c_void_p), 0)
    _check1d(ctx, rc)


def af1d_step(ctx, dt_out=None):
    if dt_out is False:
        _check1d(ctx, _lib().af1d_step(ctx, None, 0))
        return None
    d = C.c_double()
    _check1d(ctx, _lib().af1d_step(ctx, C.cast(C.byref(d), C.c_void_p), 0))
    return d.value


def af1d_status(ctx, reset: bool = False):
    cnt = (C.c_longlong * AF_NSTAT)()
    rc = _lib().af1d_status(ctx, cnt, int(reset))
    return rc, dict(zip(STAT_NAMES, [int(v) for v in cnt]))


def af1d_timing(ctx, enable: bool):
    """Per-kernel event timing of the 1D stages, as af_timing (names k1_* and k_dt)."""
    if enable:
        _check1d(ctx, _lib().af1d_timing(ctx, 1, None, None))
        return None
    ms = (C.c_double * len(KERNEL_NAMES))()
    n = (C.c_longlong * len(KERNEL_NAMES))()
    _check1d(ctx, _lib().af1d_timing(ctx, 0, C.cast(ms, C.c_void_p), C.cast(n, C.c_void_p)))
    return {(k if k == "k_dt" else k.replace("k_", "k1_")): (ms[i], int(n[i])) for i, k in enumerate(KERNEL_NAMES)}


def af1d_last_error(ctx) -> str:
    return _lib().af1d_last_error(ctx).decode()


def af1d_destroy(ctx) -> None:
    if ctx:
        _lib().af1d_destroy(ctx)


class Solver1D:
    """A 1D run (af1d_*): n cells, gamma, periodic or outflow, on [x0, x1]."""

    def __init__(self, n: int, gamma: float, bc: int = AF_BC_PERIODIC, domain=(0.0, 1.0), cfl: float = 0.2,
                 kappa: float = 0.0, pp_on: bool = True, stream=None):
        self.ctx = af1d_create(n, gamma, bc)
        af1d_set_domain(self.ctx, domain[0], domain[1])
        af1d_set_params(self.ctx, cfl, kappa, pp_on)
        if stream is not None:
            af1d_set_stream(self.ctx, stream)

    def set_state(self, U):
        af1d_set_state(self.ctx, U)

    def get_state(self, out=None, device: bool = True):
        return af1d_get_state(self.ctx, out, device)

    def get_stage(self, out=None, device: bool = True):
        return af1d_get_stage(self.ctx, out, device)

    def dt(self):
        return af1d_dt(self.ctx)

    def stage(self, s: int, dt=None):
        af1d_stage(self.ctx, s, dt)

    def step(self, dt_out=None):
        return af1d_step(self.ctx, dt_out)

    def status(self, reset: bool = False):
        return af1d_status(self.ctx, reset)

    def timing(self, enable: bool):
        return af1d_timing(self.ctx, enable)

    def close(self):
        if self.ctx:
            af1d_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
