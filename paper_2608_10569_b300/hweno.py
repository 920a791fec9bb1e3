"""Thin ctypes binding of libhweno.so (C ABI in include/hweno.h).

Every function of the C ABI is exposed under the same name with the same
arguments; ``Solver`` wraps a handle for torch tensors and numpy arrays.  This
module only marshals arguments: every step of the method runs in the CUDA
library, and importing fails loudly if the library is missing.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libhweno.so")

HWENO_OK = 0
HWENO_ERR_ARG = -1
HWENO_ERR_CUDA = -2
HWENO_ERR_INADMISSIBLE = -3
HWENO_ERR_NONFINITE = -4
HWENO_ERR_TIMEOUT = -5
HWENO_ERR_STATE = -6
HWENO_FP64 = 0
HWENO_MIXED = 1
HWENO_SCHEME_GR = 0
HWENO_SCHEME_DR = 1
HWENO_SOURCE_NONE = 0
HWENO_SOURCE_MMS52 = 1
BC = {"periodic": 0, "noslip": 1, "symmetry": 2, "slip": 3, "inflow": 4, "outflow": 5}
SCHEME = {"gr": HWENO_SCHEME_GR, "dr": HWENO_SCHEME_DR, HWENO_SCHEME_GR: HWENO_SCHEME_GR,
          HWENO_SCHEME_DR: HWENO_SCHEME_DR}
SOURCE = {None: HWENO_SOURCE_NONE, "none": HWENO_SOURCE_NONE, "mms52": HWENO_SOURCE_MMS52,
          HWENO_SOURCE_NONE: HWENO_SOURCE_NONE, HWENO_SOURCE_MMS52: HWENO_SOURCE_MMS52}

# kernel indices of hweno_profile_read
KERNELS = ["ghost", "cons_recon", "face_moments", "weak_moments", "grad_recon", "flux", "assemble",
           "rk_update", "source"]


class HwenoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("hweno error %d: %s" % (code, msg))
        self.code = code


class hweno_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("Re", ctypes.c_double),
                ("bc", ctypes.c_int * 4),
                ("cfl", ctypes.c_double), ("b_visc", ctypes.c_double),
                ("eps_pp", ctypes.c_double), ("eps_weno", ctypes.c_double),
                ("max_halvings", ctypes.c_int), ("precision", ctypes.c_int),
                ("scheme", ctypes.c_int), ("source", ctypes.c_int),
                ("inflow", ((ctypes.c_double * 4) * 2) * 4), ("band", (ctypes.c_double * 2) * 4),
                ("linear_grad", ctypes.c_int), ("pad_", ctypes.c_int)]


class hweno_diag(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt_last", ctypes.c_double),
                ("alpha_star", ctypes.c_double), ("beta_max", ctypes.c_double),
                ("pp_active", ctypes.c_double), ("cell_stages", ctypes.c_double),
                ("min_rho", ctypes.c_double), ("min_p", ctypes.c_double),
                ("totals", ctypes.c_double * 4),
                ("steps", ctypes.c_longlong), ("rejected", ctypes.c_longlong),
                ("fp64_steps", ctypes.c_longlong), ("max_kinetic_share", ctypes.c_double)]


class hweno1d_config(ctypes.Structure):
    """include/hweno1d.h: one problem of the one-dimensional solver (Sec. 2)"""
    _fields_ = [("n", ctypes.c_int), ("bc", ctypes.c_int * 2), ("scheme", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("Re", ctypes.c_double),
                ("cfl", ctypes.c_double), ("b_visc", ctypes.c_double),
                ("eps_pp", ctypes.c_double), ("eps_weno", ctypes.c_double),
                ("max_halvings", ctypes.c_int), ("source", ctypes.c_int),
                ("inflow", (ctypes.c_double * 3) * 2)]


BC1D = {"periodic": 0, "reflective": 1, "inflow": 2, "outflow": 3}


_lib = None

# (name, restype, argtypes) of every exported entry point
_H = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
SIGNATURES = [
    ("hweno_config_default", ctypes.c_int, [ctypes.POINTER(hweno_config)]),
    ("hweno_init", ctypes.c_int, [ctypes.POINTER(hweno_config), ctypes.c_void_p, ctypes.POINTER(_H)]),
    ("hweno_destroy", None, [_H]),
    ("hweno_last_error", ctypes.c_char_p, [_H]),
    ("hweno_set_state", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int]),
    ("hweno_set_time", ctypes.c_int, [_H, ctypes.c_double]),
    ("hweno_get_state", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int]),
    ("hweno_residual", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("hweno_step", ctypes.c_int, [_H, ctypes.c_double, _D, ctypes.POINTER(ctypes.c_int)]),
    ("hweno_advance", ctypes.c_int, [_H, ctypes.c_double, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_int)]),
    ("hweno_get_diag", ctypes.c_int, [_H, ctypes.POINTER(hweno_diag)]),
    ("hweno_debug_fields", ctypes.c_int, [_H, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    ("hweno_profile", ctypes.c_int, [_H, ctypes.c_int]),
    ("hweno_profile_read", ctypes.c_int, [_H, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong), _D]),
    ("hweno_launch_count", ctypes.c_longlong, [_H]),
    ("hweno_measure_peak", ctypes.c_int, [_H, ctypes.c_int, _D]),
    ("hweno_residual_noalloc", ctypes.c_int, [ctypes.POINTER(hweno_config), ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("hweno_adjoint_init", ctypes.c_int, [_H]),
    ("hweno_adjoint_residual", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, _D, ctypes.c_int]),
    ("hweno_adjoint_reserve", ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int]),
    ("hweno_adjoint_record", ctypes.c_int, [_H, ctypes.c_int]),
    ("hweno_adjoint_replay", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, _D, ctypes.c_int]),
    ("hweno_adjoint_segment", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int, _D, ctypes.c_void_p,
                                             ctypes.c_void_p, _D, ctypes.c_int]),
    ("hweno_adjoint_step", ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                          ctypes.c_void_p, _D, ctypes.c_int]),
    ("hweno_batch_init", ctypes.c_int, [ctypes.POINTER(hweno_config), ctypes.c_int, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    ("hweno_batch_destroy", None, [ctypes.c_void_p]),
    ("hweno_batch_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("hweno_batch_case", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(_H)]),
    ("hweno_batch_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("hweno_batch_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    ("hweno_batch_launch_count", ctypes.c_longlong, [ctypes.c_void_p]),
    ("hweno1d_config_default", ctypes.c_int, [ctypes.POINTER(hweno1d_config)]),
    ("hweno1d_advance", ctypes.c_int, [ctypes.POINTER(hweno1d_config), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_void_p), ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, _D, ctypes.c_void_p]),
    ("hweno1d_step", ctypes.c_int, [ctypes.POINTER(hweno1d_config), ctypes.c_void_p, ctypes.c_double,
                                    ctypes.c_double, _D, ctypes.c_void_p]),
    ("hweno1d_residual", ctypes.c_int, [ctypes.POINTER(hweno1d_config), ctypes.c_void_p, ctypes.c_double,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("hweno1d_last_error", ctypes.c_char_p, []),
]


def load(path=LIB_PATH):
    """Load libhweno.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError("libhweno.so not found at %s: build it with "
                              "`python -m paper_2608_10569_b300.build` (there is no CPU fallback)" % path)
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def __getattr__(name):
    # hweno_* attributes resolve to the raw C entry points
    if name.startswith("hweno_"):
        return getattr(load(), name)
    raise AttributeError(name)


def _check(h, rc):
    if rc != HWENO_OK:
        msg = load().hweno_last_error(h)
        raise HwenoError(rc, msg.decode() if msg else "")
    return rc


def make_config(nx, ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, gamma=1.4, Pr=0.72, Re=1000.0,
                bc=("periodic",) * 4, cfl=0.6, b_visc=1e-3, eps_pp=1e-12, eps_weno=1e-8,
                max_halvings=60, precision="fp64", scheme="gr", source=0, inflow=None, band=None,
                linear_grad=False, **_ignored):
    """inflow: per face (xlo, xhi, ylo, yhi) None or the pair of conserved states (inside,
    outside) the face's band; band: per face None or (centre, half width)"""
    c = hweno_config()
    load().hweno_config_default(ctypes.byref(c))
    c.nx, c.ny = int(nx), int(ny)
    c.x0, c.x1, c.y0, c.y1 = float(x0), float(x1), float(y0), float(y1)
    c.gamma, c.Pr, c.Re = float(gamma), float(Pr), float(Re)
    for k in range(4):
        c.bc[k] = BC[bc[k]] if isinstance(bc[k], str) else int(bc[k])
    c.cfl, c.b_visc, c.eps_pp, c.eps_weno = float(cfl), float(b_visc), float(eps_pp), float(eps_weno)
    c.max_halvings = int(max_halvings)
    c.precision = HWENO_MIXED if precision in ("mixed", HWENO_MIXED) else HWENO_FP64
    c.scheme = SCHEME[scheme]
    c.source = SOURCE[source]
    for k in range(4):
        if inflow and inflow[k] is not None:
            for a in range(2):
                for v in range(4):
                    c.inflow[k][a][v] = float(inflow[k][a][v])
        if band and band[k] is not None:
            c.band[k][0], c.band[k][1] = float(band[k][0]), float(band[k][1])
    c.linear_grad = 1 if linear_grad else 0
    return c


def _ptr_of(a, count=None):
    """(pointer, on_device) of a torch tensor or numpy array: contiguous float64, with
    exactly count elements when count is given (the library reads or writes that many,
    so a shorter buffer is refused here rather than overrun)."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("need a C-contiguous float64 array")
        n, out = a.size, (ctypes.c_void_p(a.ctypes.data), 0)
    else:
        import torch
        if not isinstance(a, torch.Tensor):
            raise TypeError("need a numpy array or a torch tensor")
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("need a contiguous float64 tensor")
        n, out = a.numel(), (ctypes.c_void_p(a.data_ptr()), (1 if a.is_cuda else 0))
    if count is not None and n != count:
        raise ValueError("need %d float64 elements, got %d" % (count, n))
    return out


class Solver:
    """One HWENO-GR solver instance on the current CUDA device."""

    def __init__(self, case_params, precision="fp64", stream=None):
        import torch
        self.lib = load()
        p = dict(case_params)
        p["precision"] = precision
        self.cfg = make_config(**p)
        self.nx, self.ny = self.cfg.nx, self.cfg.ny
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = _H()
        rc = self.lib.hweno_init(ctypes.byref(self.cfg), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if rc != HWENO_OK:
            raise HwenoError(rc, self.lib.hweno_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.hweno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, q):
        ptr, dev = _ptr_of(q, 12 * self.nx * self.ny)
        _check(self.h, self.lib.hweno_set_state(self.h, ptr, dev))

    def set_time(self, t):
        _check(self.h, self.lib.hweno_set_time(self.h, float(t)))

    def get_state(self, out=None):
        import torch
        if out is None:
            out = torch.empty((12, self.ny, self.nx), dtype=torch.float64, device="cuda")
        ptr, dev = _ptr_of(out, 12 * self.nx * self.ny)
        _check(self.h, self.lib.hweno_get_state(self.h, ptr, dev))
        return out

    def residual(self, rhs=None, vhat=None):
        import torch
        if rhs is None:
            rhs = torch.empty((12, self.ny, self.nx), dtype=torch.float64, device="cuda")
        if vhat is None:
            vhat = torch.empty((8, self.ny, self.nx), dtype=torch.float64, device="cuda")
        pr, dr = _ptr_of(rhs, 12 * self.nx * self.ny)
        pv, dv = _ptr_of(vhat, 8 * self.nx * self.ny)
        if dr != dv:
            raise ValueError("rhs and vhat must both be host or both be device buffers")
        _check(self.h, self.lib.hweno_residual(self.h, pr, pv, dr))
        return rhs, vhat

    def step(self, dt=0.0):
        used = ctypes.c_double(0.0)
        rej = ctypes.c_int(0)
        _check(self.h, self.lib.hweno_step(self.h, float(dt), ctypes.byref(used), ctypes.byref(rej)))
        return used.value, rej.value

    def advance(self, t_end, max_steps=2 ** 31 - 1):
        t = ctypes.c_double(0.0)
        n = ctypes.c_int(0)
        _check(self.h, self.lib.hweno_advance(self.h, float(t_end), int(max_steps), ctypes.byref(t),
                                              ctypes.byref(n)))
        return t.value, n.value

    def diag(self):
        d = hweno_diag()
        _check(self.h, self.lib.hweno_get_diag(self.h, ctypes.byref(d)))
        return {"t": d.t, "dt_last": d.dt_last, "alpha_star": d.alpha_star, "beta_max": d.beta_max,
                "pp_active": d.pp_active, "cell_stages": d.cell_stages, "min_rho": d.min_rho,
                "min_p": d.min_p, "totals": list(d.totals), "steps": d.steps, "rejected": d.rejected,
                "fp64_steps": d.fp64_steps, "max_kinetic_share": d.max_kinetic_share}

    def debug_fields(self, which):
        import torch
        n = {0: 48, 1: 36, 2: 18, 3: 126, 4: 2}[which]
        out = torch.empty((n, self.ny, self.nx), dtype=torch.float64, device="cuda")
        ptr, dev = _ptr_of(out, n * self.nx * self.ny)
        _check(self.h, self.lib.hweno_debug_fields(self.h, int(which), ptr, dev))
        return out

    def profile(self, enable=True):
        _check(self.h, self.lib.hweno_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        out = {}
        for k, name in enumerate(KERNELS):
            n = ctypes.c_longlong(0)
            ms = ctypes.c_double(0.0)
            _check(self.h, self.lib.hweno_profile_read(self.h, k, ctypes.byref(n), ctypes.byref(ms)))
            out[name] = (n.value, ms.value)
        return out

    def launch_count(self):
        return self.lib.hweno_launch_count(self.h)

    def adjoint_init(self):
        _check(self.h, self.lib.hweno_adjoint_init(self.h))

    def adjoint_residual(self, x, rbar=None, mbar=None, xbar=None):
        """(xbar, mubar): VJP of (residual, modified moments) at the state x."""
        if xbar is None:
            xbar = np.zeros_like(x) if isinstance(x, np.ndarray) else x.new_empty(x.shape)
        n12, n8 = 12 * self.nx * self.ny, 8 * self.nx * self.ny
        px, dx = _ptr_of(x, n12)
        po, _ = _ptr_of(xbar, n12)
        pr = _ptr_of(rbar, n12)[0] if rbar is not None else None
        pm = _ptr_of(mbar, n8)[0] if mbar is not None else None
        mub = ctypes.c_double(0.0)
        _check(self.h, self.lib.hweno_adjoint_residual(self.h, px, pr, pm, po, ctypes.byref(mub), dx))
        return xbar, mub.value

    def adjoint_reserve(self, max_steps, keep_intermediates=True):
        rc = self.lib.hweno_adjoint_reserve(self.h, int(max_steps), 1 if keep_intermediates else 0)
        if rc < 0:
            _check(self.h, rc)
        return rc == 1

    def adjoint_record(self, on=True):
        _check(self.h, self.lib.hweno_adjoint_record(self.h, 1 if on else 0))

    def adjoint_replay(self, lam_end, lam_start=None):
        """(lam_start, mubar) through the recorded steps."""
        import torch
        if lam_start is None:
            lam_start = torch.empty_like(lam_end) if torch.is_tensor(lam_end) else np.empty_like(lam_end)
        pl, dl = _ptr_of(lam_end, 12 * self.nx * self.ny)
        po, do = _ptr_of(lam_start, 12 * self.nx * self.ny)
        if dl != do:
            raise ValueError("lam_end and lam_start must both be host or both be device buffers")
        mub = ctypes.c_double(0.0)
        _check(self.h, self.lib.hweno_adjoint_replay(self.h, pl, po, ctypes.byref(mub), dl))
        return lam_start, mub.value

    def adjoint_segment(self, q_start, dts, lam_end, lam_start=None):
        """(lam_start, mubar) through the steps with sizes dts from q_start."""
        import torch
        if lam_start is None:
            lam_start = torch.empty_like(lam_end)
        n12 = 12 * self.nx * self.ny
        pq, dq = _ptr_of(q_start, n12)
        pl, dl = _ptr_of(lam_end, n12)
        po, do = _ptr_of(lam_start, n12)
        if not (dq == dl == do):
            raise ValueError("q_start, lam_end and lam_start must all be host or all be device buffers")
        arr = (ctypes.c_double * len(dts))(*[float(x) for x in dts])
        mub = ctypes.c_double(0.0)
        _check(self.h, self.lib.hweno_adjoint_segment(self.h, pq, len(dts), arr, pl, po, ctypes.byref(mub), dq))
        return lam_start, mub.value

    def adjoint_step(self, q, dt, lam_next, lam=None):
        """(lam, mubar): the VJP of the SSP-RK3 step q -> q' taken with dt (mu = 1/Re)."""
        import torch
        if lam is None:
            lam = torch.empty_like(lam_next)
        n12 = 12 * self.nx * self.ny
        pq, dq = _ptr_of(q, n12)
        pl, dl = _ptr_of(lam_next, n12)
        po, do = _ptr_of(lam, n12)
        if not (dq == dl == do):
            raise ValueError("q, lam_next and lam must all be host or all be device buffers")
        mub = ctypes.c_double(0.0)
        _check(self.h, self.lib.hweno_adjoint_step(self.h, pq, float(dt), pl, po, ctypes.byref(mub), dq))
        return lam, mub.value

    def measure_peak(self, which):
        """FP64 (which=0) or FP32 (which=1) FMA throughput in TFLOP/s."""
        tf = ctypes.c_double(0.0)
        _check(self.h, self.lib.hweno_measure_peak(self.h, int(which), ctypes.byref(tf)))
        return tf.value


class _CaseView(Solver):
    """A case of a Batch: the Solver interface on a handle the batch owns."""

    def __init__(self, lib, h, cfg):
        self.lib = lib
        self.h = h
        self.cfg = cfg
        self.nx, self.ny = cfg.nx, cfg.ny

    def close(self):
        self.h = None  # owned by the batch


class Batch:
    """An ensemble of independent problems advanced together (hweno_batch_*)."""

    def __init__(self, case_params_list, precision="mixed", stream=None):
        self.lib = load()
        n = len(case_params_list)
        cfgs = (hweno_config * n)()
        for k, p in enumerate(case_params_list):
            p = dict(p)
            p["precision"] = precision
            cfgs[k] = make_config(**p)
        self.cfgs = cfgs
        b = ctypes.c_void_p()
        s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        rc = self.lib.hweno_batch_init(cfgs, n, s, ctypes.byref(b))
        if rc != HWENO_OK:
            raise HwenoError(rc, self.lib.hweno_last_error(None).decode())
        self.b = b
        self.cases = []
        for k in range(n):
            h = _H()
            self._check(self.lib.hweno_batch_case(self.b, k, ctypes.byref(h)))
            self.cases.append(_CaseView(self.lib, h, cfgs[k]))

    def _check(self, rc):
        if rc != HWENO_OK:
            raise HwenoError(rc, self.lib.hweno_batch_last_error(self.b).decode())

    def step(self, nsteps=1):
        rej = ctypes.c_int(0)
        self._check(self.lib.hweno_batch_step(self.b, int(nsteps), ctypes.byref(rej)))
        return rej.value

    def autotune(self):
        chosen = (ctypes.c_int * 6)()
        self._check(self.lib.hweno_batch_autotune(self.b, chosen))
        return list(chosen)

    def launch_count(self):
        return self.lib.hweno_batch_launch_count(self.b)

    def close(self):
        if getattr(self, "b", None):
            for c in self.cases:
                c.close()
            self.lib.hweno_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _rollout_autograd():
    import torch
    from torch.autograd.function import once_differentiable

    class Rollout(torch.autograd.Function):
        """q_T = Phi^n(q_0) for n SSP-RK3 steps of the FP64 solver, differentiable with
        respect to the initial state q_0 and the viscosity mu = 1/Re.

        Forward: the steps under the time-step rule of Sec. 5; the step sizes are kept,
        the state is checkpointed every `ckpt` steps, and (when a gradient will be taken)
        the final segment is recorded with its stage states and intermediates
        (hweno_adjoint_record).  Backward: the adjoint of the final segment from the
        recording (hweno_adjoint_replay), then for each earlier segment, last to first,
        one recomputation from its checkpoint with the kept step sizes followed by the
        reverse sweep (hweno_adjoint_segment).  The step sizes are held fixed."""

        @staticmethod
        def forward(ctx, q0, mu, case_params, nsteps, ckpt, record):
            p = dict(case_params)
            p["Re"] = 1.0 / float(mu)
            s = Solver(p, precision="fp64")
            s.set_state(q0.detach().contiguous())
            dts, ckpts = [], {0: q0.detach().clone()}
            last = ((nsteps - 1) // ckpt) * ckpt if nsteps > 0 else 0  # first step of the final segment
            recorded = False
            for n in range(nsteps):
                if record and n == last:
                    s.adjoint_init()
                    s.adjoint_reserve(min(ckpt, nsteps), keep_intermediates=True)
                    s.adjoint_record(True)
                    recorded = True
                dt, _ = s.step()
                dts.append(dt)
                if (n + 1) % ckpt == 0 and n + 1 < nsteps:
                    ckpts[n + 1] = s.get_state().clone()
            if recorded:
                s.adjoint_record(False)
            qT = s.get_state().clone()
            if not record:  # no gradient will be taken: release the device memory now
                s.close()
                s = None
            ctx.solver = s
            ctx.dts = dts
            ctx.ckpts = ckpts
            ctx.ckpt = ckpt
            ctx.recorded = last if recorded else None
            return qT

        @staticmethod
        @once_differentiable
        def backward(ctx, qbar):
            s = ctx.solver
            if s is None:
                raise RuntimeError("hweno.rollout: a second backward through the same rollout; its solver "
                                   "was released by the first (run the rollout again)")
            ctx.solver = None
            dts, ckpts, K = ctx.dts, ctx.ckpts, ctx.ckpt
            n = len(dts)
            if ctx.recorded is None:
                # nothing recorded in the forward: storage for the recomputed segments.
                # A forward that recorded reserved it already, and reserving again could
                # drop its recording
                s.adjoint_init()
                s.adjoint_reserve(min(K, n), keep_intermediates=True)
            lam = qbar.detach().contiguous().clone()
            mubar = 0.0
            for a in reversed(sorted(ckpts)):
                b = min(a + K, n)
                if a == ctx.recorded:
                    lam, mb = s.adjoint_replay(lam)
                else:
                    lam, mb = s.adjoint_segment(ckpts[a], dts[a:b], lam)
                mubar += mb
            s.close()
            return lam, qbar.new_tensor(mubar), None, None, None, None

    return Rollout


def rollout(q0, mu, case_params, nsteps, ckpt=20):
    """Differentiable n-step FP64 rollout; see the Rollout autograd function."""
    import torch
    global _ROLLOUT
    if "_ROLLOUT" not in globals():
        _ROLLOUT = _rollout_autograd()
    if not torch.is_tensor(mu):
        mu = torch.tensor(float(mu), dtype=torch.float64, device=q0.device)
    record = torch.is_grad_enabled() and (q0.requires_grad or mu.requires_grad)
    return _ROLLOUT.apply(q0, mu, case_params, int(nsteps), int(ckpt), bool(record))


# ---------------------------------------------------------------------------
# one-dimensional solver (include/hweno1d.h)

def make_config1d(n, x0=0.0, x1=1.0, gamma=1.4, Pr=0.72, Re=1000.0, bc=("periodic", "periodic"), cfl=0.6,
                  b_visc=1e-3, eps_pp=1e-12, eps_weno=1e-8, max_halvings=60, scheme="gr", source=0,
                  inflow=((0.0, 0.0, 0.0), (0.0, 0.0, 0.0)), **_ignored):
    c = hweno1d_config()
    load().hweno1d_config_default(ctypes.byref(c))
    c.n = int(n)
    for k in range(2):
        c.bc[k] = BC1D[bc[k]] if isinstance(bc[k], str) else int(bc[k])
    c.x0, c.x1 = float(x0), float(x1)
    c.gamma, c.Pr, c.Re = float(gamma), float(Pr), float(Re)
    c.cfl, c.b_visc, c.eps_pp, c.eps_weno = float(cfl), float(b_visc), float(eps_pp), float(eps_weno)
    c.max_halvings = int(max_halvings)
    c.scheme = SCHEME[scheme]
    c.source = {None: 0, "none": 0, "mms51": 1, 0: 0, 1: 1}[source]
    for k in range(2):
        for v in range(3):
            c.inflow[k][v] = float(inflow[k][v])
    return c


def _dev1d(a, count):
    """device pointer of a CUDA float64 tensor of count elements (the 1D ABI takes device
    buffers only)"""
    ptr, dev = _ptr_of(a, count)
    if not dev:
        raise ValueError("the 1D solver takes CUDA tensors")
    return ptr


def _check1d(rc):
    if rc != HWENO_OK:
        raise HwenoError(rc, load().hweno1d_last_error().decode())


def advance1d(params_list, states, t0, t_end, max_steps=2 ** 31 - 1, stream=None):
    """Advance several 1D problems together (one thread block each) from t0 to t_end.
    states: CUDA float64 tensors of shape (6, n_k), updated in place.  Returns one
    dict per problem: t, steps, rejections, status, pp_active (limiter activations)."""
    lib = load()
    n = len(params_list)
    cfgs = (hweno1d_config * n)(*[make_config1d(**p) for p in params_list])
    if len(states) != n:
        raise ValueError("one state per problem: %d problems, %d states" % (n, len(states)))
    ptrs = (ctypes.c_void_p * n)(*[_dev1d(q, 6 * cfgs[k].n).value for k, q in enumerate(states)])
    out = np.zeros(5 * n)
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check1d(lib.hweno1d_advance(cfgs, n, ptrs, float(t0), float(t_end), int(max_steps),
                                 out.ctypes.data_as(_D), s))
    return [{"t": out[5 * k], "steps": int(out[5 * k + 1]), "rejections": int(out[5 * k + 2]),
             "status": int(out[5 * k + 3]), "pp_active": int(out[5 * k + 4])} for k in range(n)]


def step1d(params, state, t, dt=0.0, stream=None):
    """One SSP-RK3 step of a 1D problem (state a CUDA (6, n) tensor, in place)."""
    lib = load()
    c = make_config1d(**params)
    out = np.zeros(4)
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check1d(lib.hweno1d_step(ctypes.byref(c), _dev1d(state, 6 * c.n), float(t), float(dt),
                              out.ctypes.data_as(_D), s))
    return {"dt": out[0], "rejections": int(out[1]), "status": int(out[2]), "pp_active": int(out[3])}


def residual1d(params, state, t=0.0, stream=None):
    """Eq. (2.2) at state (CUDA (6, n) tensor) and time t: (rhs (6, n), vhat (3, n))."""
    import torch
    lib = load()
    c = make_config1d(**params)
    rhs = torch.empty((6, c.n), dtype=torch.float64, device="cuda")
    vhat = torch.empty((3, c.n), dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check1d(lib.hweno1d_residual(ctypes.byref(c), _dev1d(state, 6 * c.n), float(t), _dev1d(rhs, 6 * c.n),
                                  _dev1d(vhat, 3 * c.n), s))
    return rhs, vhat
