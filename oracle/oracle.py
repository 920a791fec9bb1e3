"""ctypes front-end of the FP64 CPU oracles (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It compiles ``hweno_oracle.c`` with gcc
(no FMA contraction, OpenMP over cells) into ``liboracle.so`` beside it, and the same
source over dual numbers (``hweno_oracle_jvp.cpp``, g++) into ``liboracle_jvp.so``:
the forward-mode tangents ``residual_jvp`` and ``step_jvp``.

States are numpy float64 arrays of shape (12, ny, nx): plane 4*m + v holds
moment m (0 = cell average, 1 = scaled xi-moment, 2 = scaled eta-moment) of
conserved variable v (rho, rho*u, rho*v, E).

The one-dimensional oracle (``hweno1d_oracle.c``, the scheme of Sec. 2) is in the same
library, behind the ``*1d`` functions: its states are arrays of shape (6, n), plane
3*m + v holding moment m (0 average, 1 scaled moment) of v (rho, rho*u, E).
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hweno_oracle.c")
_SRC1 = os.path.join(_HERE, "hweno1d_oracle.c")
_HDR = os.path.join(_HERE, "oracle_tables.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_JVP_SRC = os.path.join(_HERE, "hweno_oracle_jvp.cpp")
_JVP_LIB = os.path.join(_HERE, "liboracle_jvp.so")
_CNT_SRC = os.path.join(_HERE, "hweno_oracle_count.cpp")
_CNT_LIB = os.path.join(_HERE, "liboracle_count.so")
_lock = threading.Lock()
_lib = None
_jvp = None
_cnt = None

BC = {"periodic": 0, "noslip": 1, "symmetry": 2, "slip": 3, "inflow": 4, "outflow": 5}
# viscous gradients: HWENO-GR (weak-derivative moments) or HWENO-DR (differentiated
# convective candidates, the comparison scheme)
SCHEME = {"gr": 0, "dr": 1, 0: 0, 1: 1}
# source terms: none, or Example 5.2's manufactured source
SOURCE = {None: 0, "none": 0, "mms52": 1, 0: 0, 1: 1}


class _Cfg(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("Re", ctypes.c_double),
                ("bc", ctypes.c_int * 4),
                ("cfl", ctypes.c_double), ("b_visc", ctypes.c_double),
                ("eps_pp", ctypes.c_double), ("eps_weno", ctypes.c_double),
                ("max_halvings", ctypes.c_int), ("linear_weights", ctypes.c_int),
                ("limiter", ctypes.c_int), ("scheme", ctypes.c_int),
                ("source", ctypes.c_int), ("pad2_", ctypes.c_int), ("time", ctypes.c_double),
                ("inflow", ((ctypes.c_double * 4) * 2) * 4), ("band", (ctypes.c_double * 2) * 4),
                ("linear_grad", ctypes.c_int), ("pad3_", ctypes.c_int)]


def build(force=False):
    """Compile the oracle shared library if it is missing or stale."""
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR),
                                          os.path.getmtime(_SRC1)))
    if force or stale:
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", "-o", _LIB + ".tmp", _SRC, _SRC1, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    stale = (not os.path.exists(_JVP_LIB) or
             os.path.getmtime(_JVP_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR),
                                               os.path.getmtime(_JVP_SRC)))
    if force or stale:
        # -fpermissive -w: the C source assigns malloc/calloc results without casts,
        # the only construct C++ rejects; nothing else is diagnosed
        cmd = ["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-std=c++17", "-fpermissive", "-w", "-o", _JVP_LIB + ".tmp", _JVP_SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_JVP_LIB + ".tmp", _JVP_LIB)
    stale = (not os.path.exists(_CNT_LIB) or
             os.path.getmtime(_CNT_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR),
                                               os.path.getmtime(_CNT_SRC)))
    if force or stale:
        # serial (no OpenMP): the counters are plain globals
        cmd = ["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-std=c++17", "-fpermissive", "-w", "-o", _CNT_LIB + ".tmp", _CNT_SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_CNT_LIB + ".tmp", _CNT_LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.or_residual.argtypes = [ctypes.POINTER(_Cfg), dp, dp, dp, dp, dp, dp, dp, dp, dp]
            lib.or_residual_cells.argtypes = [ctypes.POINTER(_Cfg), dp, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int), dp, dp]
            lib.or_step.argtypes = [ctypes.POINTER(_Cfg), dp, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, dp]
            lib.or_advance.argtypes = [ctypes.POINTER(_Cfg), dp, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, dp]
            lib.or_fill_ghosts.argtypes = [ctypes.POINTER(_Cfg), dp, dp]
            lib.or_hweno_scalar.argtypes = [dp, ctypes.c_double, ctypes.c_int, dp, dp, dp, dp, dp]
            lib.or_mms_source_export.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_double, dp]
            lib.or_hweno_scalar_dr.argtypes = [dp, ctypes.c_double, ctypes.c_int, dp, dp]
            lib.or_theta_root_export.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double]
            lib.or_theta_root_export.restype = ctypes.c_double
            lib.or_eigen_export.argtypes = [dp, ctypes.c_double, ctypes.c_int, dp, dp]
            _bind_wave_bound(lib)
            _lib = lib
    return _lib


def _bind_wave_bound(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    lib.or_wave_bound_export.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int, dp, dp]
    lib.or_wave_bound_export.restype = ctypes.c_double


def wave_bound(cfg, direction, s, gr, lib=None):
    """max(|u_n| + c, PP wave-speed bound of Eq. (3.3)) at one face-point state: s the
    conserved state (4), gr = (u_x, u_y, v_x, v_y, e_x, e_y); lib: a library built from
    this source (default: the oracle's own)"""
    lib = lib or _load()
    s = np.ascontiguousarray(s, dtype=float)
    gr = np.ascontiguousarray(gr, dtype=float)
    return lib.or_wave_bound_export(ctypes.byref(cfg), int(direction), _ptr(s), _ptr(gr))


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_cfg(nx, ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, gamma=1.4, Pr=0.72, Re=1000.0,
             bc=("periodic",) * 4, cfl=0.6, b_visc=1e-3, eps_pp=1e-12, eps_weno=1e-8,
             max_halvings=60, linear_weights=False, limiter=True, scheme="gr", source=0, time=0.0,
             inflow=None, band=None, linear_grad=False, **_ignored):
    """inflow: per side (xlo, xhi, ylo, yhi) None or a pair of conserved states (A, B);
    band: per side (centre, half-width) of the face coordinate where A applies"""
    c = _Cfg()
    c.nx, c.ny = int(nx), int(ny)
    c.x0, c.x1, c.y0, c.y1 = float(x0), float(x1), float(y0), float(y1)
    c.gamma, c.Pr, c.Re = float(gamma), float(Pr), float(Re)
    for k in range(4):
        c.bc[k] = BC[bc[k]] if isinstance(bc[k], str) else int(bc[k])
    c.cfl, c.b_visc, c.eps_pp, c.eps_weno = float(cfl), float(b_visc), float(eps_pp), float(eps_weno)
    c.max_halvings = int(max_halvings)
    c.linear_weights = 1 if linear_weights else 0
    c.limiter = 1 if limiter else 0
    c.scheme = SCHEME[scheme]
    c.source = SOURCE[source]
    c.time = float(time)
    c.linear_grad = 1 if linear_grad else 0
    for k in range(4):
        st = inflow[k] if inflow and inflow[k] is not None else None
        if c.bc[k] == 4 and st is None:
            raise ValueError("an inflow side needs its states")
        if st is not None:
            for a in range(2):
                for v in range(4):
                    c.inflow[k][a][v] = float(st[a][v])
        if band and band[k] is not None:
            c.band[k][0], c.band[k][1] = float(band[k][0]), float(band[k][1])
    mirror = any(c.bc[k] != 0 for k in range(4))
    if mirror and (c.nx < 4 or c.ny < 4):
        raise ValueError("mirror boundaries need at least 4 cells per direction")
    if (c.bc[0] == 0) != (c.bc[1] == 0) or (c.bc[2] == 0) != (c.bc[3] == 0):
        raise ValueError("periodic boundaries must be set on both sides")
    return c


def _state(cfg, q):
    q = np.ascontiguousarray(q, dtype=np.float64)
    if q.shape != (12, cfg.ny, cfg.nx):
        raise ValueError(f"state shape {q.shape} != (12, {cfg.ny}, {cfg.nx})")
    return q


def residual(cfg, q, dumps=False):
    """Spatial operator: returns dict(rhs (12,ny,nx), vhat (8,ny,nx), diag) and,
    with dumps, the intermediate fields face (48,..), vol (36,..), rm (18,..),
    grad (126,..), theta (2,..)."""
    lib = _load()
    q = _state(cfg, q)
    ny, nx = cfg.ny, cfg.nx
    out = {"rhs": np.zeros((12, ny, nx)), "vhat": np.zeros((8, ny, nx)), "diag": np.zeros(8)}
    d = {}
    if dumps:
        d = {"face": np.zeros((48, ny, nx)), "vol": np.zeros((36, ny, nx)),
             "rm": np.zeros((18, ny, nx)), "grad": np.zeros((126, ny, nx)),
             "theta": np.zeros((2, ny, nx))}
    rc = lib.or_residual(ctypes.byref(cfg), _ptr(q), _ptr(out["rhs"]), _ptr(out["vhat"]),
                         _ptr(out["diag"]), _ptr(d.get("face")), _ptr(d.get("vol")),
                         _ptr(d.get("rm")), _ptr(d.get("grad")), _ptr(d.get("theta")))
    if rc:
        raise MemoryError("oracle residual failed")
    out.update(d)
    return out


def residual_cells(cfg, q, ci, cj):
    """Residual of selected cells: returns rhs (n,12), vhat (n,8)."""
    lib = _load()
    q = _state(cfg, q)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    cj = np.ascontiguousarray(cj, dtype=np.int32)
    n = len(ci)
    rhs, vh = np.zeros((n, 12)), np.zeros((n, 8))
    rc = lib.or_residual_cells(ctypes.byref(cfg), _ptr(q), n,
                               ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               cj.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(rhs), _ptr(vh))
    if rc:
        raise MemoryError("oracle residual_cells failed")
    return rhs, vh


def step(cfg, q, t=0.0, t_end=np.inf, dt_fixed=0.0):
    """One SSP-RK3 step; returns (q_new, stats dict)."""
    lib = _load()
    q = _state(cfg, q).copy()
    st = np.zeros(6)
    lib.or_step(ctypes.byref(cfg), _ptr(q), float(t), float(t_end), float(dt_fixed), _ptr(st))
    return q, {"dt": st[0], "rejections": int(st[1]), "alpha": st[2], "beta_max": st[3],
               "pp_active": st[4], "status": int(st[5])}


def advance(cfg, q, t0, t_end, max_steps=10 ** 9):
    lib = _load()
    q = _state(cfg, q).copy()
    st = np.zeros(10)
    lib.or_advance(ctypes.byref(cfg), _ptr(q), float(t0), float(t_end), int(max_steps), _ptr(st))
    return q, {"dt": st[0], "status": int(st[5]), "t": st[6], "steps": int(st[7]),
               "rejections": int(st[8]), "pp_active": st[9]}


def fill_ghosts(cfg, q):
    lib = _load()
    q = _state(cfg, q)
    out = np.zeros((12, cfg.ny + 8, cfg.nx + 8))
    lib.or_fill_ghosts(ctypes.byref(cfg), _ptr(q), _ptr(out))
    return out


def hweno_scalar(d17, eps=1e-8, linear=False):
    """One scalar reconstruction: dict(pts (21,), mom (2,), beta (5,), omega (5,), c0 (15,))."""
    lib = _load()
    d17 = np.ascontiguousarray(d17, dtype=np.float64)
    assert d17.shape == (17,)
    o = {"pts": np.zeros(21), "mom": np.zeros(2), "beta": np.zeros(5), "omega": np.zeros(5),
         "c0": np.zeros(15)}
    lib.or_hweno_scalar(_ptr(d17), float(eps), 1 if linear else 0, _ptr(o["pts"]), _ptr(o["mom"]),
                        _ptr(o["beta"]), _ptr(o["omega"]), _ptr(o["c0"]))
    return o


def hweno_scalar_dr(d17, eps=1e-8, linear=False):
    """HWENO-DR derivatives of one scalar reconstruction: (d/dxi (21,), d/deta (21,)) at
    the 12 face and 9 volume points, in scaled units."""
    lib = _load()
    d17 = np.ascontiguousarray(d17, dtype=np.float64)
    assert d17.shape == (17,)
    dxi, deta = np.zeros(21), np.zeros(21)
    lib.or_hweno_scalar_dr(_ptr(d17), float(eps), 1 if linear else 0, _ptr(dxi), _ptr(deta))
    return dxi, deta


def mms_source(cfg, x, y, t):
    """Example 5.2's source S(x, y, t) (4,) at one point."""
    lib = _load()
    S = np.zeros(4)
    lib.or_mms_source_export(ctypes.byref(cfg), float(x), float(y), float(t), _ptr(S))
    return S


def theta_root(ub, uq, eps, gamma):
    lib = _load()
    ub = np.ascontiguousarray(ub, dtype=np.float64)
    uq = np.ascontiguousarray(uq, dtype=np.float64)
    return lib.or_theta_root_export(_ptr(ub), _ptr(uq), float(eps), float(gamma))


def eigen(ub, gamma, direction):
    lib = _load()
    ub = np.ascontiguousarray(ub, dtype=np.float64)
    L, R = np.zeros((4, 4)), np.zeros((4, 4))
    lib.or_eigen_export(_ptr(ub), float(gamma), int(direction), _ptr(L), _ptr(R))
    return L, R


def _load_jvp():
    global _jvp
    _load()
    with _lock:
        if _jvp is None:
            lib = ctypes.CDLL(_JVP_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.or_jvp_residual.argtypes = [ctypes.POINTER(_Cfg), dp, dp, ctypes.c_double, dp, dp, dp, dp]
            lib.or_jvp_step.argtypes = [ctypes.POINTER(_Cfg), dp, dp, ctypes.c_double, ctypes.c_double, dp]
            _jvp = lib
    return _jvp


def residual_jvp(cfg, q, qdot=None, dmu=0.0):
    """The residual and its tangent along (qdot, dmu) by the dual-number build:
    dict(rhs, rhs_dot (12,ny,nx), vhat, vhat_dot (8,ny,nx)).  dmu is the tangent of
    mu = 1/Re."""
    lib = _load_jvp()
    q = _state(cfg, q)
    qd = None if qdot is None else _state(cfg, qdot)
    ny, nx = cfg.ny, cfg.nx
    o = {"rhs": np.zeros((12, ny, nx)), "rhs_dot": np.zeros((12, ny, nx)),
         "vhat": np.zeros((8, ny, nx)), "vhat_dot": np.zeros((8, ny, nx))}
    rc = lib.or_jvp_residual(ctypes.byref(cfg), _ptr(q), _ptr(qd), float(dmu), _ptr(o["rhs"]),
                             _ptr(o["rhs_dot"]), _ptr(o["vhat"]), _ptr(o["vhat_dot"]))
    if rc:
        raise MemoryError("oracle residual_jvp failed")
    return o


def step_jvp(cfg, q, qdot, dt, dmu=0.0):
    """One SSP-RK3 step of size dt and its tangent along (qdot, dmu), by the
    dual-number build: returns (q_new, qdot_new, stats dict)."""
    lib = _load_jvp()
    q = _state(cfg, q).copy()
    qd = _state(cfg, qdot).copy()
    st = np.zeros(6)
    lib.or_jvp_step(ctypes.byref(cfg), _ptr(q), _ptr(qd), float(dmu), float(dt), _ptr(st))
    return q, qd, {"dt": st[0], "rejections": int(st[1]), "alpha": st[2], "beta_max": st[3],
                   "pp_active": st[4], "status": int(st[5])}


# ---------------------------------------------------------------------------
# one-dimensional scheme (Sec. 2)

BC1 = {"periodic": 0, "reflective": 1, "inflow": 2, "outflow": 3}


class _Cfg1(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("bc", ctypes.c_int * 2), ("pad0_", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("Re", ctypes.c_double),
                ("cfl", ctypes.c_double), ("b_visc", ctypes.c_double),
                ("eps_pp", ctypes.c_double), ("eps_weno", ctypes.c_double),
                ("max_halvings", ctypes.c_int), ("linear_weights", ctypes.c_int),
                ("limiter", ctypes.c_int), ("scheme", ctypes.c_int), ("source", ctypes.c_int),
                ("pad1_", ctypes.c_int), ("time", ctypes.c_double),
                ("inflow", (ctypes.c_double * 3) * 2)]


_lib1_ready = False


def _load1():
    global _lib1_ready
    lib = _load()
    with _lock:
        if not _lib1_ready:
            dp = ctypes.POINTER(ctypes.c_double)
            P = ctypes.POINTER(_Cfg1)
            lib.or1_residual.argtypes = [P, dp, dp, dp, dp, dp, dp, dp]
            lib.or1_step.argtypes = [P, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
            lib.or1_advance.argtypes = [P, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp]
            lib.or1_hweno_scalar.argtypes = [dp, ctypes.c_double, ctypes.c_int, dp, dp, dp, dp, dp, dp]
            lib.or1_mms_source_export.argtypes = [P, ctypes.c_double, ctypes.c_double, dp]
            _lib1_ready = True
    return lib


def make_cfg1d(n, x0=0.0, x1=1.0, gamma=1.4, Pr=0.72, Re=1000.0, bc=("periodic", "periodic"), cfl=0.6,
               b_visc=1e-3, eps_pp=1e-12, eps_weno=1e-8, max_halvings=60, linear_weights=False, limiter=True,
               scheme="gr", source=0, time=0.0, inflow=((0.0, 0.0, 0.0), (0.0, 0.0, 0.0)), **_ignored):
    c = _Cfg1()
    c.n = int(n)
    for k in range(2):
        c.bc[k] = BC1[bc[k]] if isinstance(bc[k], str) else int(bc[k])
    if (c.bc[0] == 0) != (c.bc[1] == 0):
        raise ValueError("periodic boundaries must be set on both sides")
    c.x0, c.x1 = float(x0), float(x1)
    c.gamma, c.Pr, c.Re = float(gamma), float(Pr), float(Re)
    c.cfl, c.b_visc, c.eps_pp, c.eps_weno = float(cfl), float(b_visc), float(eps_pp), float(eps_weno)
    c.max_halvings = int(max_halvings)
    c.linear_weights = 1 if linear_weights else 0
    c.limiter = 1 if limiter else 0
    c.scheme = SCHEME[scheme]
    c.source = {None: 0, "none": 0, "mms51": 1, 0: 0, 1: 1}[source]
    c.time = float(time)
    for k in range(2):
        for v in range(3):
            c.inflow[k][v] = float(inflow[k][v])
    return c


def _state1(cfg, q):
    q = np.ascontiguousarray(q, dtype=np.float64)
    if q.shape != (6, cfg.n):
        raise ValueError(f"state shape {q.shape} != (6, {cfg.n})")
    return q


def residual1d(cfg, q, dumps=False):
    """Sec. 2's spatial operator: dict(rhs (6,n), vhat (3,n), diag) and, with dumps,
    pts (12,n) (Lobatto point 3*g + v, limited), grad (8,n) (2*g + (u_x, e_x)),
    theta (2,n)."""
    lib = _load1()
    q = _state1(cfg, q)
    n = cfg.n
    out = {"rhs": np.zeros((6, n)), "vhat": np.zeros((3, n)), "diag": np.zeros(8)}
    d = {}
    if dumps:
        d = {"pts": np.zeros((12, n)), "grad": np.zeros((8, n)), "theta": np.zeros((2, n))}
    rc = lib.or1_residual(ctypes.byref(cfg), _ptr(q), _ptr(out["rhs"]), _ptr(out["vhat"]), _ptr(out["diag"]),
                          _ptr(d.get("pts")), _ptr(d.get("grad")), _ptr(d.get("theta")))
    if rc:
        raise MemoryError("oracle 1D residual failed")
    out.update(d)
    return out


def step1d(cfg, q, t=0.0, t_end=np.inf, dt_fixed=0.0):
    lib = _load1()
    q = _state1(cfg, q).copy()
    st = np.zeros(6)
    lib.or1_step(ctypes.byref(cfg), _ptr(q), float(t), float(t_end), float(dt_fixed), _ptr(st))
    return q, {"dt": st[0], "rejections": int(st[1]), "alpha": st[2], "beta_max": st[3],
               "pp_active": st[4], "status": int(st[5])}


def advance1d(cfg, q, t0, t_end, max_steps=10 ** 9):
    lib = _load1()
    q = _state1(cfg, q).copy()
    st = np.zeros(10)
    lib.or1_advance(ctypes.byref(cfg), _ptr(q), float(t0), float(t_end), int(max_steps), _ptr(st))
    return q, {"dt": st[0], "pp_active": st[4], "status": int(st[5]), "t": st[6], "steps": int(st[7]),
               "rejections": int(st[8])}


def hweno_scalar1d(d5, eps=1e-8, linear=False):
    """One 1D scalar reconstruction (Appendix A.1): dict(pts (4,), dpts (4,), mom, beta (3,),
    omega (3,), c0 (5,)) at the four Lobatto points, derivatives in scaled units."""
    lib = _load1()
    d5 = np.ascontiguousarray(d5, dtype=np.float64)
    assert d5.shape == (5,)
    o = {"pts": np.zeros(4), "dpts": np.zeros(4), "mom": np.zeros(1), "beta": np.zeros(3),
         "omega": np.zeros(3), "c0": np.zeros(5)}
    lib.or1_hweno_scalar(_ptr(d5), float(eps), 1 if linear else 0, _ptr(o["pts"]), _ptr(o["dpts"]),
                         _ptr(o["mom"]), _ptr(o["beta"]), _ptr(o["omega"]), _ptr(o["c0"]))
    o["mom"] = float(o["mom"][0])
    return o


def mms_source1d(cfg, x, t):
    lib = _load1()
    S = np.zeros(3)
    lib.or1_mms_source_export(ctypes.byref(cfg), float(x), float(t), _ptr(S))
    return S


# ---------------------------------------------------------------------------
# operation counts (hweno_oracle_count.cpp): the oracle's state-dependent, non-trivial
# floating-point operations, by kind
OP_KINDS = ("add", "mul", "div", "sqrt", "trans")
PHASES = ("traces", "limiter", "weak_moments", "gradients", "face_fluxes", "balances", "alpha")


def _load_cnt():
    global _cnt
    with _lock:
        if _cnt is None:
            build()
            lib = ctypes.CDLL(_CNT_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            lp = ctypes.POINTER(ctypes.c_longlong)
            lib.or_count_phases.argtypes = [ctypes.POINTER(_Cfg), dp, lp]
            lib.or_count_call.argtypes = [ctypes.POINTER(_Cfg), dp, ctypes.c_int, ctypes.c_double, lp]
            lib.or_count_theta_root.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, lp]
            lib.or_count_theta_root.restype = ctypes.c_double
            lib.or_count_hweno.argtypes = [dp, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, dp, lp]
            _cnt = lib
    return _cnt


def _counts(a):
    return dict(zip(OP_KINDS, (int(x) for x in a)))


def op_count_phases(cfg, q):
    """{phase: {kind: count}} of one residual (phases PHASES), each distinct computation
    counted once, where it first occurs"""
    lib = _load_cnt()
    q = _state(cfg, q)
    out = np.zeros(len(PHASES) * len(OP_KINDS), dtype=np.int64)
    if lib.or_count_phases(ctypes.byref(cfg), _ptr(q), out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))):
        raise RuntimeError("or_count_phases failed")
    return {p: _counts(out[k * len(OP_KINDS):(k + 1) * len(OP_KINDS)]) for k, p in enumerate(PHASES)}


def op_count_call(cfg, q, what, dt=0.0):
    """counts of a whole call: what = "residual" (with diagnostics), "residual_nodiag",
    or "step" (one SSP-RK3 step of size dt)"""
    lib = _load_cnt()
    q = _state(cfg, q)
    out = np.zeros(len(OP_KINDS), dtype=np.int64)
    code = {"residual": 0, "residual_nodiag": 1, "step": 2}[what]
    if lib.or_count_call(ctypes.byref(cfg), _ptr(q), code, float(dt),
                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))):
        raise RuntimeError("or_count_call failed")
    return _counts(out)


def op_count_theta_root(ub, uq, eps, gamma):
    lib = _load_cnt()
    ub = np.ascontiguousarray(ub, dtype=float)
    uq = np.ascontiguousarray(uq, dtype=float)
    out = np.zeros(len(OP_KINDS), dtype=np.int64)
    t = lib.or_count_theta_root(_ptr(ub), _ptr(uq), float(eps), float(gamma),
                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
    return t, _counts(out)


def op_count_hweno(d17, points, eps=1e-8, linear=False):
    """(build counts, evaluation counts) of one scalar reconstruction and its values at
    the points [(xi, eta), ...]"""
    lib = _load_cnt()
    d = np.ascontiguousarray(d17, dtype=float)
    pts = np.asarray(points, dtype=float).reshape(-1, 2)
    xi = np.ascontiguousarray(pts[:, 0])
    eta = np.ascontiguousarray(pts[:, 1])
    out = np.zeros(2 * len(OP_KINDS), dtype=np.int64)
    lib.or_count_hweno(_ptr(d), float(eps), int(bool(linear)), len(pts), _ptr(xi), _ptr(eta),
                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
    return _counts(out[:len(OP_KINDS)]), _counts(out[len(OP_KINDS):])


def flops(counts):
    """floating-point operations of a count record: additions, multiplications,
    divisions and square roots one each (transcendentals kept apart)"""
    return counts["add"] + counts["mul"] + counts["div"] + counts["sqrt"]


def algorithmic_flops(cfg, q):
    """algorithmic floating-point work of the method per cell and RK stage, by phase of
    the spatial operator plus the stage update: the distinct state-dependent operations
    of the oracle on the state q, on a periodic grid (every ghost cell a copy, so no halo
    is counted; see hweno_oracle_count.cpp), divided by the number of cells.  Returns
    {phase: flops per cell} with the phases PHASES and "stage_update" (the SSP-RK3
    combination and the admissibility check)."""
    assert all(b == BC["periodic"] for b in cfg.bc), "counts per cell need a periodic grid"
    n = cfg.nx * cfg.ny
    out = {p: flops(c) / n for p, c in op_count_phases(cfg, q).items()}
    with_diag = flops(op_count_call(cfg, q, "residual"))
    step = flops(op_count_call(cfg, q, "step", dt=1e-6))
    out["stage_update"] = (step - 3 * with_diag) / (3 * n)
    return out
