"""ctypes binding of the CPU FP64 oracle (af_oracle.cpp).

TEST INFRASTRUCTURE ONLY: the test-suite, __graft_entry__.smoke() and the
benchmark's CPU-baseline / reference arm are the only users.  The product
(paper_2506_04857_gb300) never imports this package.

States are lists of four float64 arrays [8, nyp, nxp] (cell averages, x-face,
y-face and corner point values; see af_inputs for the layout).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "af_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIBS = {}
_LOCK = threading.Lock()

NSTATS = 12
STAT_NAMES = ["src_limited", "lambda_lt1", "face_theta_lt1", "sensor_lt099", "newton_solves", "newton_maxit",
              "shrink", "point_limited", "cfl_violations", "center_limited", "nonadmissible", "cell_shrink"]
PHASES = ["dt", "pointdata", "center", "point_ho", "point_pp", "sensor_phi", "sensor_theta", "face", "cell_src",
          "cell_update", "cell_final", "rk"]
KINDS = ["add", "mul", "div", "sqrt", "exp", "minmax", "cmp"]


class Coeffs(C.Structure):
    """or_coeffs: the limiter coefficients of one stage (see af_oracle.cpp)."""
    _fields_ = [("ths_x", C.POINTER(C.c_double)), ("ths_y", C.POINTER(C.c_double)),
                ("ths_c", C.POINTER(C.c_double)), ("th_src", C.POINTER(C.c_double)),
                ("lam", C.POINTER(C.c_double)), ("th_x", C.POINTER(C.c_double)),
                ("th_y", C.POINTER(C.c_double)), ("th_pt", C.POINTER(C.c_double) * 4)]


COEFF_NAMES = ["ths_x", "ths_y", "ths_c", "th_src", "lam", "th_x", "th_y", "th_pt0", "th_pt1", "th_pt2", "th_pt3"]


def coeff_shapes(nx, ny, bc):
    """Array shapes of the stage coefficients (faces, cells, scaling-limiter theta*/theta** per class)."""
    from af_inputs import class_extents
    ext = class_extents(nx, ny, bc)
    sh = {"ths_x": (ext[1][1], ext[1][0]), "ths_y": (ext[2][1], ext[2][0]), "ths_c": (ny, nx), "th_src": (ny, nx),
          "lam": (4, ny, nx), "th_x": (ext[1][1], ext[1][0]), "th_y": (ext[2][1], ext[2][0])}
    for c in range(4):
        sh["th_pt%d" % c] = (2, ext[c][1], ext[c][0])
    return sh


def _coeffs_struct(arrs):
    cs = Coeffs()
    for name in COEFF_NAMES[:7]:
        setattr(cs, name, _dp(arrs[name]) if name in arrs else None)
    for c in range(4):
        key = "th_pt%d" % c
        cs.th_pt[c] = _dp(arrs[key]) if key in arrs else None
    return cs


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double),
                ("y1", C.c_double), ("cfl", C.c_double), ("kappa", C.c_double), ("bc", C.c_int),
                ("pp_on", C.c_int), ("src_cell_on", C.c_int), ("src_point_on", C.c_int),
                ("side", C.c_int * 4), ("inflow_lo", C.c_double), ("inflow_hi", C.c_double),
                ("inflow_U", C.c_double * 8), ("src_point_upwind", C.c_int)]


def params_for(pb, kappa=None, pp_on=True, src_cell_on=True, src_point_on=True, cfl=None,
               src_point_upwind=False) -> Params:
    P = Params(pb.gamma, pb.x0, pb.x1, pb.y0, pb.y1, pb.cfl if cfl is None else cfl,
               pb.kappa if kappa is None else kappa, pb.bc, int(pp_on), int(src_cell_on), int(src_point_on))
    sides = getattr(pb, "sides", (0, 0, 0, 0))
    for k in range(4):
        P.side[k] = int(sides[k])
    P.inflow_lo = float(getattr(pb, "inflow_lo", 0.0))
    P.inflow_hi = float(getattr(pb, "inflow_hi", 0.0))
    inU = getattr(pb, "inflow_U", None)
    for k in range(8):
        P.inflow_U[k] = float(inU[k]) if inU is not None else 0.0
    P.src_point_upwind = int(src_point_upwind)
    return P


def build(force: bool = False) -> None:
    """Compile the oracle (plain and counting builds) with g++."""
    os.makedirs(_BUILD, exist_ok=True)
    jobs = [("liboracle.so", ["-fopenmp"]), ("liboracle_count.so", ["-DAF_ORACLE_COUNT"]),
            ("liboracle_cs.so", ["-DAF_ORACLE_COMPLEX"])]
    procs = []
    for name, extra in jobs:
        out = os.path.join(_BUILD, name)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        tmp = out + ".tmp%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", *extra, "-o", tmp, _SRC]
        procs.append((subprocess.Popen(cmd), tmp, out))
    for p, tmp, out in procs:
        if p.wait() != 0:
            raise RuntimeError("oracle build failed")
        os.replace(tmp, out)


def _lib(count: bool = False, complex_step: bool = False):
    key = "cs" if complex_step else ("count" if count else "plain")
    name = {"cs": "liboracle_cs.so", "count": "liboracle_count.so", "plain": "liboracle.so"}[key]
    with _LOCK:
        if key not in _LIBS:
            build()
            lib = C.CDLL(os.path.join(_BUILD, name))
            pp = C.POINTER(C.POINTER(C.c_double))
            dp = C.POINTER(C.c_double)
            lib.or_dt.restype = C.c_double
            lib.or_dt.argtypes = [C.POINTER(Params), C.c_int, C.c_int, pp]
            lib.or_stage.argtypes = [C.POINTER(Params), C.c_int, C.c_int, pp, pp, C.c_double, C.c_double, C.c_double,
                                     pp, C.POINTER(C.c_longlong)]
            lib.or_step.argtypes = [C.POINTER(Params), C.c_int, C.c_int, pp, C.c_double, dp, C.POINTER(C.c_longlong)]
            lib.or_rhs.argtypes = [C.POINTER(Params), C.c_int, C.c_int, pp, pp]
            lib.or_flux.argtypes = [C.c_int, dp, C.c_double, dp]
            lib.or_pressure.restype = C.c_double
            lib.or_pressure.argtypes = [dp, C.c_double]
            lib.or_fast_speed.restype = C.c_double
            lib.or_fast_speed.argtypes = [C.c_int, dp, C.c_double]
            lib.or_spectral_radius.restype = C.c_double
            lib.or_spectral_radius.argtypes = [C.c_int, dp, C.c_double]
            lib.or_llf_flux.restype = C.c_double
            lib.or_llf_flux.argtypes = [C.c_int, dp, dp, C.c_double, dp]
            lib.or_center_value.argtypes = [dp, dp, dp, dp]
            lib.or_fd.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, dp]
            lib.or_flux_limiter.restype = C.c_int
            lib.or_flux_limiter.argtypes = [dp, dp, C.c_double, C.c_double, C.c_double, dp, C.POINTER(C.c_int)]
            lib.or_scaling_limiter.argtypes = [dp, dp, C.c_double, dp, dp]
            lib.or_sensor_phi.argtypes = [dp, dp, dp, dp, dp, C.c_double, C.c_double, C.c_double, dp]
            lib.or_sensor.argtypes = [C.POINTER(Params), C.c_int, C.c_int, pp, dp, dp]
            lib.or_divb.argtypes = [C.POINTER(Params), C.c_int, C.c_int, pp, dp]
            lib.or1d_dt.restype = C.c_double
            lib.or1d_dt.argtypes = [C.POINTER(Params), C.c_int, pp]
            lib.or1d_stage.argtypes = [C.POINTER(Params), C.c_int, pp, pp, C.c_double, C.c_double, C.c_double, pp,
                                       C.POINTER(C.c_longlong)]
            lib.or1d_step.argtypes = [C.POINTER(Params), C.c_int, pp, C.c_double, dp, C.POINTER(C.c_longlong)]
            lib.or_stage_rec.argtypes = [C.POINTER(Params), C.c_int, C.c_int, pp, pp, C.c_double, C.c_double,
                                         C.c_double, pp, C.POINTER(C.c_longlong), C.POINTER(Coeffs),
                                         C.POINTER(Coeffs)]
            if key == "cs":
                lib.or_stage_cs.argtypes = [C.POINTER(Params), C.c_int, C.c_int, pp, pp, pp, pp, C.c_double,
                                            C.c_double, C.c_double, pp, pp, C.POINTER(Coeffs)]
                lib.or_step_cs.restype = C.c_int
                lib.or_step_cs.argtypes = [C.POINTER(Params), C.c_int, C.c_int, pp, pp, C.c_double]
            lib.or_counts.restype = C.c_int
            lib.or_counts.argtypes = [C.POINTER(C.c_longlong), C.c_int]
            _LIBS[key] = lib
        return _LIBS[key]


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ptrs(U: List[np.ndarray]):
    arr = (C.POINTER(C.c_double) * 4)(*[_dp(u) for u in U])
    return arr


def _check(U, nx, ny, bc):
    from af_inputs import class_extents
    ext = class_extents(nx, ny, bc)
    out = []
    for c in range(4):
        a = np.ascontiguousarray(U[c], dtype=np.float64)
        if a.shape != (8, ext[c][1], ext[c][0]):
            raise ValueError("class %d has shape %s, expected %s" % (c, a.shape, (8, ext[c][1], ext[c][0])))
        out.append(a)
    return out


def _empty(nx, ny, bc):
    from af_inputs import class_extents
    return [np.zeros((8, e[1], e[0])) for e in class_extents(nx, ny, bc)]


def dt(pb, U, count=False, **kw) -> float:
    P = params_for(pb, **kw)
    U = _check(U, pb.nx, pb.ny, pb.bc)
    return _lib(count).or_dt(C.byref(P), pb.nx, pb.ny, _ptrs(U))


def stage(pb, Un, Us, dt_, a, b, stats: Optional[np.ndarray] = None, count=False, **kw):
    P = params_for(pb, **kw)
    Un = _check(Un, pb.nx, pb.ny, pb.bc)
    Us = _check(Us, pb.nx, pb.ny, pb.bc)
    out = _empty(pb.nx, pb.ny, pb.bc)
    st = np.zeros(NSTATS, dtype=np.int64) if stats is None else stats
    _lib(count).or_stage(C.byref(P), pb.nx, pb.ny, _ptrs(Un), _ptrs(Us), dt_, a, b, _ptrs(out),
                         st.ctypes.data_as(C.POINTER(C.c_longlong)))
    return out


def stage_record(pb, Un, Us, dt_, a, b, stats: Optional[np.ndarray] = None, frozen: Optional[dict] = None, **kw):
    """One stage (as stage()) that also returns the limiter coefficients it took, as a dict of
    arrays (coeff_shapes).  With frozen (such a dict) the stage uses those coefficients instead
    of forming them.  Entries a stage does not form (face theta with PP limiting off) stay NaN."""
    P = params_for(pb, **kw)
    Un = _check(Un, pb.nx, pb.ny, pb.bc)
    Us = _check(Us, pb.nx, pb.ny, pb.bc)
    out = _empty(pb.nx, pb.ny, pb.bc)
    st = np.zeros(NSTATS, dtype=np.int64) if stats is None else stats
    rec = {k: np.full(v, np.nan) for k, v in coeff_shapes(pb.nx, pb.ny, pb.bc).items()}
    rs = _coeffs_struct(rec)
    fz = None
    if frozen is not None:
        frozen = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in frozen.items()}
        fz_struct = _coeffs_struct(frozen)
        fz = C.byref(fz_struct)
    _lib().or_stage_rec(C.byref(P), pb.nx, pb.ny, _ptrs(Un), _ptrs(Us), dt_, a, b, _ptrs(out),
                        st.ctypes.data_as(C.POINTER(C.c_longlong)), C.byref(rs), fz)
    return out, rec


def stage_complex(pb, Un_re, Un_im, Us_re, Us_im, dt_, a, b, frozen: Optional[dict] = None, **kw):
    """One stage a Un + b FE(Us) of complex states (complex-step differentiation) with the
    limiter coefficients frozen at `frozen` (a stage_record dict) or formed from the complex
    state (None).  Returns (re, im)."""
    P = params_for(pb, **kw)
    arrs = [_check(u, pb.nx, pb.ny, pb.bc) for u in (Un_re, Un_im, Us_re, Us_im)]
    re, im = _empty(pb.nx, pb.ny, pb.bc), _empty(pb.nx, pb.ny, pb.bc)
    fz = None
    if frozen is not None:
        frozen = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in frozen.items()}
        fz_struct = _coeffs_struct(frozen)
        fz = C.byref(fz_struct)
    _lib(complex_step=True).or_stage_cs(C.byref(P), pb.nx, pb.ny, *[_ptrs(u) for u in arrs], dt_, a, b,
                                        _ptrs(re), _ptrs(im), fz)
    return re, im


def step(pb, U, dt_in: float = 0.0, stats: Optional[np.ndarray] = None, count=False, **kw):
    """One SSP-RK3 step; returns (new state, dt used)."""
    P = params_for(pb, **kw)
    V = [a.copy() for a in _check(U, pb.nx, pb.ny, pb.bc)]
    st = np.zeros(NSTATS, dtype=np.int64) if stats is None else stats
    d = C.c_double(0.0)
    _lib(count).or_step(C.byref(P), pb.nx, pb.ny, _ptrs(V), dt_in, C.byref(d),
                        st.ctypes.data_as(C.POINTER(C.c_longlong)))
    return V, d.value


def rhs(pb, U, **kw):
    P = params_for(pb, **kw)
    U = _check(U, pb.nx, pb.ny, pb.bc)
    out = _empty(pb.nx, pb.ny, pb.bc)
    _lib().or_rhs(C.byref(P), pb.nx, pb.ny, _ptrs(U), _ptrs(out))
    return out


def sensor(pb, U, **kw):
    """theta^s at x-faces [ny, nxf] and y-faces [nyf, nx] of the state U."""
    from af_inputs import class_extents
    P = params_for(pb, **kw)
    U = _check(U, pb.nx, pb.ny, pb.bc)
    ext = class_extents(pb.nx, pb.ny, pb.bc)
    tx = np.zeros((ext[1][1], ext[1][0]))
    ty = np.zeros((ext[2][1], ext[2][0]))
    _lib().or_sensor(C.byref(P), pb.nx, pb.ny, _ptrs(U), _dp(tx), _dp(ty))
    return tx, ty


def divb(pb, U, count=False, **kw):
    """(divB_1, divB_2): the two discrete divergence measures of Example 4.4 (node
    divergences of the bi-parabola; Simpson edge integral of B.n per cell)."""
    P = params_for(pb, **kw)
    U = _check(U, pb.nx, pb.ny, pb.bc)
    out = np.zeros(2)
    _lib(count).or_divb(C.byref(P), pb.nx, pb.ny, _ptrs(U), _dp(out))
    return float(out[0]), float(out[1])


def diagnostics(pb, U):
    """Run diagnostics of a state by their plain definitions: the minimum density
    and pressure p = (gamma-1)(E - |rho v|^2/(2 rho) - |B|^2/2) of each DoF class,
    and the total mass dx dy sum(rho_bar)."""
    U = _check(U, pb.nx, pb.ny, pb.bc)
    g = pb.gamma
    min_rho, min_p = [], []
    for u in U:
        p = (g - 1.0) * (u[7] - 0.5 * (u[1] ** 2 + u[2] ** 2 + u[3] ** 2) / u[0] - 0.5 * (u[4] ** 2 + u[5] ** 2 + u[6] ** 2))
        min_rho.append(float(u[0].min()))
        min_p.append(float(p.min()))
    return {"min_rho": min_rho, "min_p": min_p, "mass": float(U[0][0].sum()) * pb.dx * pb.dy}


# ---- the 1D scheme: states are [averages [8, n], point values [8, nf]] ----------
def _check1(U, pb):
    nf = pb.n if pb.bc == 0 else pb.n + 1
    A = np.ascontiguousarray(U[0], dtype=np.float64)
    P = np.ascontiguousarray(U[1], dtype=np.float64)
    if A.shape != (8, pb.n) or P.shape != (8, nf):
        raise ValueError("1D state must be [8, %d] and [8, %d]" % (pb.n, nf))
    return [A, P]


def dt1(pb, U, count=False, **kw) -> float:
    P = params_for(pb, **kw)
    return _lib(count).or1d_dt(C.byref(P), pb.n, _ptrs(_check1(U, pb)))


def stage1(pb, Un, Us, dt_, a, b, stats: Optional[np.ndarray] = None, count=False, **kw):
    P = params_for(pb, **kw)
    Un, Us = _check1(Un, pb), _check1(Us, pb)
    out = [np.zeros_like(Un[0]), np.zeros_like(Un[1])]
    st = np.zeros(NSTATS, dtype=np.int64) if stats is None else stats
    _lib(count).or1d_stage(C.byref(P), pb.n, _ptrs(Un), _ptrs(Us), dt_, a, b, _ptrs(out),
                      st.ctypes.data_as(C.POINTER(C.c_longlong)))
    return out


def step1(pb, U, dt_in: float = 0.0, stats: Optional[np.ndarray] = None, **kw):
    """One SSP-RK3 step of the 1D scheme; returns (new state, dt used)."""
    P = params_for(pb, **kw)
    V = [a.copy() for a in _check1(U, pb)]
    st = np.zeros(NSTATS, dtype=np.int64) if stats is None else stats
    d = C.c_double(0.0)
    _lib().or1d_step(C.byref(P), pb.n, _ptrs(V), dt_in, C.byref(d), st.ctypes.data_as(C.POINTER(C.c_longlong)))
    return V, d.value


def flux(l: int, U, gamma: float) -> np.ndarray:
    u = np.ascontiguousarray(U, dtype=np.float64)
    F = np.zeros(8)
    _lib().or_flux(l, _dp(u), gamma, _dp(F))
    return F


def pressure(U, gamma: float) -> float:
    return _lib().or_pressure(_dp(np.ascontiguousarray(U, dtype=np.float64)), gamma)


def fast_speed(l: int, U, gamma: float) -> float:
    return _lib().or_fast_speed(l, _dp(np.ascontiguousarray(U, dtype=np.float64)), gamma)


def spectral_radius(l: int, U, gamma: float) -> float:
    return _lib().or_spectral_radius(l, _dp(np.ascontiguousarray(U, dtype=np.float64)), gamma)


def llf_flux(l: int, U, V, gamma: float):
    F = np.zeros(8)
    a = _lib().or_llf_flux(l, _dp(np.ascontiguousarray(U, dtype=np.float64)),
                           _dp(np.ascontiguousarray(V, dtype=np.float64)), gamma, _dp(F))
    return F, a


def center_value(avg, faces, corners) -> np.ndarray:
    out = np.zeros(8)
    _lib().or_center_value(_dp(np.ascontiguousarray(avg, dtype=np.float64)),
                           _dp(np.ascontiguousarray(faces, dtype=np.float64)),
                           _dp(np.ascontiguousarray(corners, dtype=np.float64)), _dp(out))
    return out


def fd(a, b, c, h) -> np.ndarray:
    out = np.zeros(3)
    _lib().or_fd(a, b, c, h, _dp(out))
    return out


def flux_limiter(lim1, H, eps_rho, eps_p, gamma):
    lam = np.zeros(4)
    it = C.c_int(0)
    solves = _lib().or_flux_limiter(_dp(np.ascontiguousarray(lim1, dtype=np.float64)),
                                    _dp(np.ascontiguousarray(H, dtype=np.float64)), eps_rho, eps_p, gamma,
                                    _dp(lam), C.byref(it))
    return lam, solves, it.value


def scaling_limiter(UH, UL, gamma):
    out = np.zeros(8)
    th = np.zeros(2)
    _lib().or_scaling_limiter(_dp(np.ascontiguousarray(UH, dtype=np.float64)),
                              _dp(np.ascontiguousarray(UL, dtype=np.float64)), gamma, _dp(out), _dp(th))
    return out, th


def sensor_phi(c, e, w, n, s, gamma, dx, dy) -> np.ndarray:
    """phi_1 (x), phi_1 (y), phi_2, phi_3 of one cell from five cell averages."""
    out = np.zeros(4)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (c, e, w, n, s)]
    _lib().or_sensor_phi(*[_dp(a) for a in arrs], gamma, dx, dy, _dp(out))
    return out


def step_complex(pb, U_re, U_im, dt, **kw):
    """One SSP-RK3 step of the complex state U_re + i U_im (complex-step
    differentiation) with the fixed real dt, or with dt <= 0 the step's own dt
    of the complex state.  Returns (re, im, limiter events)."""
    P = params_for(pb, **kw)
    re = [a.copy() for a in _check(U_re, pb.nx, pb.ny, pb.bc)]
    im = [a.copy() for a in _check(U_im, pb.nx, pb.ny, pb.bc)]
    act = _lib(complex_step=True).or_step_cs(C.byref(P), pb.nx, pb.ny, _ptrs(re), _ptrs(im), dt)
    return re, im, act


def counts(reset: bool = True) -> np.ndarray:
    """Operation counts [phase, kind] of the counting build since the last reset."""
    out = np.zeros(len(PHASES) * len(KINDS), dtype=np.int64)
    _lib(count=True).or_counts(out.ctypes.data_as(C.POINTER(C.c_longlong)), int(reset))
    return out.reshape(len(PHASES), len(KINDS))


def flops(cnt: np.ndarray) -> np.ndarray:
    """Flops per phase: +, -, *, /, sqrt, exp, min/max and |.| each count one
    (comparisons that only steer branches are not counted)."""
    return cnt[:, :6].sum(axis=1)
