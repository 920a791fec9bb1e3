"""GPU parity of the inflow and outflow faces (Remark 4.1; HWENO_BC_INFLOW and
HWENO_BC_OUTFLOW) and of the rectangular benchmarks built on them (Examples 5.7 and
5.9), against the FP64 oracle, with the tolerances of the other parity tests: relative
L-infinity 1e-12 of the flux scale per residual plane, 1e-12 per step, relative L1 1e-9
after a run.  Collected after the other GPU parity tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2608_10569_b300 import hweno, inputs as I  # noqa: E402
from test_gpu_parity import (RES_TOL, flux_scale, gpu_residual, rel_l1, rel_linf, res_tol,  # noqa: E402
                             state_scale)

pytestmark = pytest.mark.gpu


def open_rough():
    """rough data entering through a banded inflow face (two states taken from the
    first column), leaving through outflow faces, a symmetry face below"""
    case, q = I.random_rough(40, 36, seed=9, bc=("inflow", "outflow", "symmetry", "outflow"), Re=200.0)
    case.inflow = ((tuple(q[:4, 18, 0]), tuple(q[:4, 5, 0])), None, None, None)
    case.band = ((0.5, 0.15), None, None, None)
    return case, q


def y_jet():
    """a jet through a band of the lower face into smooth data, outflow elsewhere"""
    case, q = I.random_smooth(33, 29, seed=10, bc=("outflow", "outflow", "inflow", "outflow"))
    a = I.conserved(1.2, 0.1, 0.8, 1.5, case.gamma)
    b = I.conserved(1.0, 0.0, 0.2, 1.0, case.gamma)
    case.inflow = (None, None, (a, b), None)
    case.band = (None, None, (0.5, 0.2), None)
    return case, q


CASES = {
    "open_rough_40x36": open_rough,
    "y_jet_33x29": y_jet,
    "outflow_box_37x29": lambda: I.random_smooth(37, 29, seed=11, bc=("outflow",) * 4),
    "mach2000_32x16": lambda: I.mach2000(32, 16),
    "sedov_24": lambda: I.sedov_2d(24),
}


def ocfg(case, **kw):
    return O.make_cfg(**dict(case.params(), **kw))


@pytest.mark.parametrize("scheme", ["gr", "dr"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_residual_parity_open_faces(name, scheme):
    case, q = CASES[name]()
    p = dict(case.params(), scheme=scheme)
    s = hweno.Solver(p)
    s.set_state(torch.from_numpy(q).cuda())
    rhs, vhat = s.residual()
    d = s.diag()
    s.close()
    o = O.residual(O.make_cfg(**p), q)
    tol = res_tol(case, q)
    assert rel_linf(rhs.cpu().numpy(), o["rhs"], flux_scale(case, q)) <= tol
    assert rel_linf(vhat.cpu().numpy(), o["vhat"], state_scale(q)) <= tol
    # the wave-speed bounds come from the same traces: the same conditioning
    assert abs(d["alpha_star"] - o["diag"][0]) <= max(1e-13, tol) * o["diag"][0]
    assert abs(d["beta_max"] - o["diag"][1]) <= max(1e-12, tol) * o["diag"][1]


def test_intermediate_fields_parity_open_faces():
    """traces, volume values, weak-derivative moments, gradients and limiter factors
    next to inflow and outflow faces"""
    case, q = open_rough()
    g = gpu_residual(case, q, dumps=(0, 1, 2, 3, 4))
    o = O.residual(ocfg(case), q, dumps=True)
    assert rel_linf(g[0], o["face"], state_scale(q)) <= RES_TOL
    assert rel_linf(g[1], o["vol"], state_scale(q)) <= RES_TOL
    assert rel_linf(g[2], o["rm"]) <= RES_TOL
    assert rel_linf(g[3], o["grad"]) <= RES_TOL
    assert np.abs(g[4] - o["theta"]).max() <= 1e-13


@pytest.mark.parametrize("name", ["open_rough_40x36", "y_jet_33x29"])
def test_mixed_precision_open_faces(name):
    """the mixed path's inflow ghosts hold the hi/lo split of the prescribed state: its
    residual stays within the mixed path's bound of the FP64 oracle"""
    case, q = CASES[name]()
    g = gpu_residual(case, q, precision="mixed")
    o = O.residual(ocfg(case), q)
    assert rel_linf(g["rhs"], o["rhs"], flux_scale(case, q)) <= 1e-5
    assert rel_linf(g["vhat"], o["vhat"], state_scale(q)) <= 1e-6


def test_step_parity_open_faces():
    """a forced and a rule step; the stages refill the inflow and outflow ghosts"""
    case, q = open_rough()
    cfg = ocfg(case)
    s = hweno.Solver(case.params())
    s.set_state(torch.from_numpy(q).cuda())
    dt, rej = s.step(1e-4)
    assert dt == 1e-4 and rej == 0
    qo, st = O.step(cfg, q, dt_fixed=1e-4)
    assert rel_linf(s.get_state().cpu().numpy(), qo, state_scale(q)) <= 1e-12
    dt2, _ = s.step()
    qo2, st2 = O.step(cfg, qo)
    assert abs(dt2 - st2["dt"]) <= 1e-13 * st2["dt"]
    assert rel_linf(s.get_state().cpu().numpy(), qo2, state_scale(q)) <= 1e-12
    s.close()


@pytest.mark.parametrize("name,precision", [("y_jet_33x29", "fp64"), ("open_rough_40x36", "fp64"),
                                            ("y_jet_33x29", "mixed")])
def test_run_parity_open_faces(name, precision):
    """20 steps under the Sec. 5 rule: relative L1 <= 1e-9 against the oracle's run at
    the same time; on the mixed path, whose wave speeds come from FP32 traces, the time
    within 1e-6 and the state within 1e-5"""
    case, q = CASES[name]()
    s = hweno.Solver(case.params(), precision=precision)
    s.set_state(torch.from_numpy(q).cuda())
    qo, st = O.advance(ocfg(case), q, 0.0, 1e9, max_steps=20)
    assert st["steps"] == 20
    for _ in range(20):
        s.step()
    fp64 = precision == "fp64"
    assert abs(s.diag()["t"] - st["t"]) <= (1e-13 if fp64 else 1e-6) * st["t"]
    assert rel_l1(s.get_state().cpu().numpy(), qo) <= (1e-9 if fp64 else 1e-5)
    s.close()


def test_mach2000_steps_and_stall():
    """Example 5.9 at 32 x 16 with the restarts capped at 20: six rule steps with the
    oracle's restarts (2, 6, 7, 15, 17, 18) and step sizes, then a step that stays
    inadmissible after 20 halvings and leaves the state at t^n, as in the oracle.  The
    jet's characteristic projection (|u|/c ~ 2e3 at the band's edges) amplifies rounding
    differences next to the inflow face: the kernels' code run on the host differs from
    the oracle by 7.9e-10 in the state and 1.0e-13 in the step sizes after these steps,
    so the states are held to the conditioning bound of the other parity tests and the
    step sizes to 1e-10"""
    case, q = I.mach2000(32, 16)
    case.max_halvings = 20
    cfg = ocfg(case)
    tol = res_tol(case, q)
    s = hweno.Solver(case.params())
    s.set_state(torch.from_numpy(q).cuda())
    qo = q
    for _ in range(6):
        qo, st = O.step(cfg, qo)
        assert st["status"] == 0
        dt, rej = s.step()
        assert rej == st["rejections"] and abs(dt - st["dt"]) <= 1e-10 * st["dt"]
        assert rel_linf(s.get_state().cpu().numpy(), qo, state_scale(q)) <= tol
    _, st = O.step(cfg, qo)
    assert st["status"] == -3
    with pytest.raises(hweno.HwenoError) as e:
        s.step()
    assert e.value.code == hweno.HWENO_ERR_INADMISSIBLE
    assert rel_linf(s.get_state().cpu().numpy(), qo, state_scale(q)) <= tol
    s.close()


def test_sedov_first_step_stalls_as_in_the_oracle():
    """Example 5.7 at 24^2 with E = 1e-12 away from the corner cell and the restarts
    capped at 20: the PP wave-speed bound (about 2.5e12) keeps the first step
    inadmissible through 20 halvings in both"""
    case, q = I.sedov_2d(24)
    case.max_halvings = 20
    _, st = O.step(ocfg(case), q)
    assert st["status"] == -3
    s = hweno.Solver(case.params())
    s.set_state(torch.from_numpy(q).cuda())
    with pytest.raises(hweno.HwenoError) as e:
        s.step()
    assert e.value.code == hweno.HWENO_ERR_INADMISSIBLE
    assert np.array_equal(s.get_state().cpu().numpy(), q)
    s.close()


def test_sedov_steps_with_the_default_halvings():
    """with the default cap (60) Sedov's first step is taken after 37 halvings (dt =
    1.5e-14) and the next ones after 27, 12 and 7, as in the oracle; the step sizes agree
    to 1e-6 and the states to the conditioning bound (E = 1e-12 away from the blast: the
    kernels' code run on the host differs from the oracle by 5.7e-6 after these steps)"""
    case, q = I.sedov_2d(24)
    cfg = ocfg(case)
    tol = res_tol(case, q)
    s = hweno.Solver(case.params())
    s.set_state(torch.from_numpy(q).cuda())
    qo, t = q, 0.0
    for expect in (37, 27, 12, 7):
        qo, st = O.step(cfg, qo, t=t)
        t += st["dt"]
        dt, rej = s.step()
        assert st["status"] == 0 and st["rejections"] == expect == rej
        assert abs(dt - st["dt"]) <= 1e-6 * st["dt"]
        assert rel_linf(s.get_state().cpu().numpy(), qo, state_scale(q)) <= tol
    s.close()


def test_adjoint_with_the_linear_gradient_ablation():
    """the adjoint of the ablated gradient reconstruction (its combination is p0
    itself): residual and step VJPs against the dual oracle run with linear_grad, to
    1e-10"""
    case, q = y_jet()
    p = dict(case.params(), linear_grad=True)
    rng = np.random.default_rng(74)
    v = rng.normal(size=q.shape) * np.abs(q).reshape(12, -1).max(1)[:, None, None]
    rbar = rng.normal(size=q.shape)
    mbar = rng.normal(size=(8,) + q.shape[1:])
    lam_next = rng.normal(size=q.shape)
    dt = 1e-3
    s = hweno.Solver(p)
    s.adjoint_init()
    xbar, mub = s.adjoint_residual(q.copy(), rbar, mbar)
    lam, _ = s.adjoint_step(q.copy(), dt, lam_next, np.zeros_like(q))
    s.close()
    cfg = O.make_cfg(**p)
    t = O.residual_jvp(cfg, q, v)
    tm = O.residual_jvp(cfg, q, None, dmu=1.0)
    assert _rel((rbar * t["rhs_dot"]).sum() + (mbar * t["vhat_dot"]).sum(), (xbar * v).sum()) <= 1e-10
    assert _rel((rbar * tm["rhs_dot"]).sum() + (mbar * tm["vhat_dot"]).sum(), mub) <= 1e-10
    _, ts, st = O.step_jvp(cfg, q, v, dt)
    assert st["status"] == 0 and st["rejections"] == 0
    assert _rel((lam_next * ts).sum(), (lam * v).sum()) <= 1e-10


def test_noalloc_with_open_faces():
    case, q = y_jet()
    lib = hweno.load()
    cfg = hweno.make_config(**case.params())
    qd = torch.from_numpy(q).cuda()
    rhs = torch.full((12, case.ny, case.nx), float("nan"), dtype=torch.float64, device="cuda")
    vhat = torch.full((8, case.ny, case.nx), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = lib.hweno_residual_noalloc(ctypes.byref(cfg), ctypes.c_void_p(qd.data_ptr()),
                                    ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(vhat.data_ptr()),
                                    ctypes.c_void_p(stream.cuda_stream))
    assert rc == hweno.HWENO_OK
    torch.cuda.synchronize()
    o = O.residual(ocfg(case), q)
    assert rel_linf(rhs.cpu().numpy(), o["rhs"], flux_scale(case, q)) <= RES_TOL
    assert rel_linf(vhat.cpu().numpy(), o["vhat"], state_scale(q)) <= RES_TOL


def _rel(a, b):
    return abs(a - b) / max(abs(a), abs(b))


@pytest.mark.parametrize("name", ["y_jet_33x29", "outflow_box_37x29"])
def test_adjoint_dot_products_with_open_faces(name):
    """the adjoint's ghost transpose returns an outflow ghost's adjoint to the edge cell
    and drops an inflow ghost's: <(rbar, mbar), J v> and <lam', J_step v> from the dual
    oracle against <xbar, v> and <J^T lam', v> from the GPU, and the derivatives in
    mu = 1/Re, to 1e-10"""
    case, q = CASES[name]()
    rng = np.random.default_rng(73)
    v = rng.normal(size=q.shape) * np.abs(q).reshape(12, -1).max(1)[:, None, None]
    rbar = rng.normal(size=q.shape)
    mbar = rng.normal(size=(8,) + q.shape[1:])
    lam_next = rng.normal(size=q.shape)
    dt = 1e-3
    s = hweno.Solver(case.params())
    s.adjoint_init()
    xbar, mub = s.adjoint_residual(q.copy(), rbar, mbar)
    lam, mub_step = s.adjoint_step(q.copy(), dt, lam_next, np.zeros_like(q))
    s.close()
    cfg = ocfg(case)
    t = O.residual_jvp(cfg, q, v)
    tm = O.residual_jvp(cfg, q, None, dmu=1.0)
    assert _rel((rbar * t["rhs_dot"]).sum() + (mbar * t["vhat_dot"]).sum(), (xbar * v).sum()) <= 1e-10
    assert _rel((rbar * tm["rhs_dot"]).sum() + (mbar * tm["vhat_dot"]).sum(), mub) <= 1e-10
    _, ts, st = O.step_jvp(cfg, q, v, dt)
    assert st["status"] == 0 and st["rejections"] == 0
    assert _rel((lam_next * ts).sum(), (lam * v).sum()) <= 1e-10
    _, tms, _ = O.step_jvp(cfg, q, np.zeros_like(q), dt, dmu=1.0)
    assert _rel((lam_next * tms).sum(), mub_step) <= 1e-10


def _residual_with(params, q, precision="fp64", dumps=()):
    s = hweno.Solver(params, precision=precision)
    s.set_state(torch.from_numpy(q).cuda())
    rhs, vhat = s.residual()
    out = {"rhs": rhs.cpu().numpy(), "vhat": vhat.cpu().numpy(), "diag": s.diag()}
    for k in dumps:
        out[k] = s.debug_fields(k).cpu().numpy()
    s.close()
    return out


@pytest.mark.parametrize("name", ["open_rough_40x36", "y_jet_33x29", "sedov_24"])
def test_linear_gradient_ablation_parity(name):
    """Remark 3.1's ablation (hweno_config.linear_grad): the gradient reconstruction with
    the linear weights, i.e. p0 itself, against the oracle's; the traces, volume values,
    weak moments and limiter factors stay those of the nonlinear run, bit for bit"""
    case, q = CASES[name]()
    p = dict(case.params(), linear_grad=True)
    g = _residual_with(p, q, dumps=(0, 1, 2, 3, 4))
    o = O.residual(O.make_cfg(**p), q)
    tol = res_tol(case, q)
    assert rel_linf(g["rhs"], o["rhs"], flux_scale(case, q)) <= tol
    assert rel_linf(g["vhat"], o["vhat"], state_scale(q)) <= tol
    assert abs(g["diag"]["beta_max"] - o["diag"][1]) <= max(1e-12, tol) * o["diag"][1]
    n = _residual_with(case.params(), q, dumps=(0, 1, 2, 3, 4))
    for k in (0, 1, 2, 4):
        assert np.array_equal(g[k], n[k]), k
    assert np.abs(g[3] - n[3]).max() > 1e-6 * np.abs(n[3]).max()


def test_linear_gradient_ablation_mixed():
    case, q = open_rough()
    p = dict(case.params(), linear_grad=True)
    g = _residual_with(p, q, precision="mixed")
    o = O.residual(O.make_cfg(**p), q)
    assert rel_linf(g["rhs"], o["rhs"], flux_scale(case, q)) <= 1e-5
    assert rel_linf(g["vhat"], o["vhat"], state_scale(q)) <= 1e-6


def test_batch_with_open_faces():
    """the batch's ghost kernel takes each case's inflow states: one step of two open-face
    cases against the oracle's step at the batch's step sizes, FP64 to 1e-12 and mixed
    to 1e-5 (the mixed residual's bound times a CFL fraction)"""
    cases = [open_rough(), y_jet()]
    for prec, bound in (("fp64", 1e-12), ("mixed", 1e-5)):
        b = hweno.Batch([c.params() for c, _ in cases], precision=prec, stream=torch.cuda.Stream())
        for k, (_, q) in enumerate(cases):
            b.cases[k].set_state(q.copy())
        b.step(1)
        for k, (case, q) in enumerate(cases):
            dt = b.cases[k].diag()["dt_last"]
            qo, st = O.step(ocfg(case), q, dt_fixed=dt)
            assert st["status"] == 0
            got = b.cases[k].get_state(np.zeros_like(q))
            assert rel_linf(got, qo, state_scale(q)) <= bound, (prec, k)
        b.close()
