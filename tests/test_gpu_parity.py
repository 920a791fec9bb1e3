"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the
same seeded inputs.

Tolerances: relative L-infinity <= 1e-12 per plane after one spatial-operator
evaluation and relative L1 <= 1e-9 after a full run.  "Relative" divides by the
larger of the plane's largest oracle magnitude and the magnitude of the terms the
plane is computed from: the inviscid fluxes of the cell averages over h for the
residual, the cell averages for traces and modified moments.  Round-off of the
two implementations is proportional to the latter, which also keeps planes that
vanish by symmetry (noise of cancelling flux differences) comparable.  Sizes span
several 32x4 thread tiles with ragged tails.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2608_10569_b300 import hweno, inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

from parity_tools import (RES_TOL, RESIDUAL_CASES, char_condition, far_from, flux_scale, oracle_floor,  # noqa: E402,F401
                          rel_l1, rel_linf, res_tol, state_scale)


def gpu_residual(case, q, precision="fp64", dumps=()):
    s = hweno.Solver(case.params(), precision=precision)
    s.set_state(torch.from_numpy(q).cuda())
    rhs, vhat = s.residual()
    out = {"rhs": rhs.cpu().numpy(), "vhat": vhat.cpu().numpy(), "diag": s.diag()}
    for w in dumps:
        out[w] = s.debug_fields(w).cpu().numpy()
    s.close()
    return out


def ocfg(case):
    return O.make_cfg(**case.params())


CASES = RESIDUAL_CASES


@pytest.mark.parametrize("name", sorted(CASES))
def test_residual_parity(name, record_property):
    """1e-12 relative to the flux scale; plane-relative, within 1e-12 or 16 x the
    oracle's own one-ulp rounding floor on the case, whichever is larger (the floor
    exceeds 1e-12 where a plane is small against the fluxes it is differenced from).
    Both figures are recorded (junit properties) beside the floor."""
    case, q = CASES[name]()
    g = gpu_residual(case, q)
    o = O.residual(ocfg(case), q)
    assert res_tol(case, q) == RES_TOL
    flux_rel = rel_linf(g["rhs"], o["rhs"], flux_scale(case, q))
    plane_rel = rel_linf(g["rhs"], o["rhs"])
    floor_plane, floor_flux = oracle_floor(case, q)
    for k, v in (("flux_rel", flux_rel), ("plane_rel", plane_rel), ("floor_plane_rel", floor_plane),
                 ("floor_flux_rel", floor_flux)):
        record_property(k, v)
    print("%s: flux-relative %.2e (floor %.2e, tol %.0e); plane-relative %.2e (floor %.2e)"
          % (name, flux_rel, floor_flux, RES_TOL, plane_rel, floor_plane))
    assert flux_rel <= RES_TOL
    assert plane_rel <= max(RES_TOL, 16 * floor_plane)
    assert rel_linf(g["vhat"], o["vhat"], state_scale(q)) <= RES_TOL
    assert abs(g["diag"]["alpha_star"] - o["diag"][0]) <= 1e-13 * o["diag"][0]
    assert abs(g["diag"]["beta_max"] - o["diag"][1]) <= 1e-12 * o["diag"][1]


def test_intermediate_fields_parity():
    """traces, volume values, weak-derivative moments, gradients and limiter factors"""
    case, q = I.random_rough(40, 36, seed=7, bc=("noslip", "symmetry", "periodic", "periodic"))
    g = gpu_residual(case, q, dumps=(0, 1, 2, 3, 4))
    o = O.residual(ocfg(case), q, dumps=True)
    assert rel_linf(g[0], o["face"], state_scale(q)) <= RES_TOL
    assert rel_linf(g[1], o["vol"], state_scale(q)) <= RES_TOL
    assert rel_linf(g[2], o["rm"]) <= RES_TOL
    assert rel_linf(g[3], o["grad"]) <= RES_TOL
    assert np.abs(g[4] - o["theta"]).max() <= 1e-13


def _far_from(mask, r):
    return far_from(mask, r)


def test_limiter_engaged_parity():
    """Near-vacuum colliding streams: the limiter clips face pressures to eps_PP, where
    the residual is ill-conditioned (the PP wave-speed bound grows like 1/e at
    e ~ 1e-12).  Cells whose 9x9 dependency square holds no limited cell match to
    1e-12, the modified moments (never limited) match everywhere, the limited face
    states keep rho, p >= eps_PP, and the set of limited cells is the oracle's."""
    case, q = I.colliding_streams(48, seed=3)
    g = gpu_residual(case, q, dumps=(0, 4))
    o = O.residual(ocfg(case), q, dumps=True)
    limited = (o["theta"][0] < 1) | (o["theta"][1] < 1)
    assert limited.any() and res_tol(case, q) > RES_TOL
    far = _far_from(limited, 4)
    assert far.any()
    tol = res_tol(case, q)
    assert rel_linf(g["rhs"], o["rhs"], flux_scale(case, q), far) <= tol
    assert rel_linf(g["vhat"], o["vhat"], state_scale(q)) <= tol
    gam = case.gamma
    face = g[0].reshape(12, 4, 48, 48)
    p = (gam - 1) * (face[:, 3] - 0.5 * (face[:, 1] ** 2 + face[:, 2] ** 2) / face[:, 0])
    assert face[:, 0].min() > 0 and p.min() >= 1e-12 - 1e-13 * np.abs(face[:, 3]).max()
    glim = (g[4][0] < 1) | (g[4][1] < 1)
    assert np.array_equal(glim, limited)


def _sample_cells(case, n, seed):
    rng = np.random.default_rng(seed)
    ci = rng.integers(0, case.nx, n)
    cj = rng.integers(0, case.ny, n)
    # always include the corners and the edges
    ci = np.concatenate([ci, [0, case.nx - 1, 0, case.nx - 1, case.nx // 2]])
    cj = np.concatenate([cj, [0, 0, case.ny - 1, case.ny - 1, case.ny // 2]])
    return ci, cj


FULL = {
    "shock_tube_1024x512": lambda: I.shock_tube(1024, 512),
    "colliding_streams_2048": lambda: I.colliding_streams(2048),
    "adjoint_tg_512": lambda: I.adjoint_taylor_green(512),
}


@pytest.mark.parametrize("name", sorted(FULL))
def test_full_size_sampled_parity(name):
    """Full workload sizes, in the launch configuration the benchmark uses; sampled
    cells checked one by one against the oracle."""
    case, q = FULL[name]()
    g = gpu_residual(case, q, dumps=(4,))
    ci, cj = _sample_cells(case, 300, 99)
    if name.startswith("shock"):
        # the diaphragm is where the residual lives: sample it densely too
        ci = np.concatenate([ci, np.full(64, case.nx // 2 - 1), np.full(64, case.nx // 2)])
        cj = np.concatenate([cj, np.arange(64) * (case.ny // 64), np.arange(64) * (case.ny // 64)])
    rhs, vh = O.residual_cells(ocfg(case), q, ci, cj)
    limited = (g[4][0] < 1) | (g[4][1] < 1)
    keep = np.array([not limited[max(0, j - 4):j + 5, max(0, i - 4):i + 5].any() for i, j in zip(ci, cj)])
    assert keep.sum() > 0.5 * len(ci)
    tol = res_tol(case, q)
    assert rel_linf(g["rhs"][:, cj, ci][:, keep], rhs.T[:, keep], flux_scale(case, q)) <= tol
    assert rel_linf(g["vhat"][:, cj, ci], vh.T, state_scale(q)) <= tol


def test_step_parity_fixed_and_rule_dt():
    case, q = I.random_rough(33, 31, seed=4, bc=("noslip", "noslip", "noslip", "symmetry"))
    cfg = ocfg(case)
    s = hweno.Solver(case.params())
    s.set_state(torch.from_numpy(q).cuda())
    dt, rej = s.step(2e-3)
    assert dt == 2e-3 and rej == 0
    qo, st = O.step(cfg, q, dt_fixed=2e-3)
    assert rel_linf(s.get_state().cpu().numpy(), qo, state_scale(q)) <= 1e-12
    dt2, _ = s.step()
    qo2, st2 = O.step(cfg, qo)
    assert abs(dt2 - st2["dt"]) <= 1e-13 * st2["dt"]
    assert rel_linf(s.get_state().cpu().numpy(), qo2, state_scale(q)) <= 1e-12
    s.close()


def test_full_run_smooth_periodic():
    """64^2 periodic flow to t = 0.1 under the Sec. 5 time-step rule (about 100
    SSP-RK3 steps): relative L1 <= 1e-9 against the oracle's run."""
    case, q = I.smooth_periodic(64)
    s = hweno.Solver(case.params())
    s.set_state(torch.from_numpy(q).cuda())
    t, n = s.advance(case.t_end)
    qo, st = O.advance(ocfg(case), q, 0.0, case.t_end)
    assert st["status"] == 0 and n == st["steps"] and abs(t - st["t"]) < 1e-15
    assert rel_l1(s.get_state().cpu().numpy(), qo) <= 1e-9
    d = s.diag()
    tot0 = q[:4].sum(axis=(1, 2)) * case.dx * case.dy
    assert np.abs(np.array(d["totals"]) - tot0).max() <= 1e-13 * np.abs(tot0).max()
    s.close()


def test_restart_on_inadmissible_stage():
    """A forced step eight times the largest stable size drives a stage of the shock
    tube inadmissible; the step is repeated from t^n with dt/2 until admissible
    (Sec. 5): three restarts, as in the oracle, and the same state."""
    case, q = I.shock_tube(64, 32)
    cfg = ocfg(case)
    s = hweno.Solver(case.params())
    s.set_state(torch.from_numpy(q).cuda())
    dt, rej = s.step(0.1)
    qo, st = O.step(cfg, q, dt_fixed=0.1)
    assert st["status"] == 0 and rej == st["rejections"] == 3
    assert dt == st["dt"] == 0.0125
    assert rel_linf(s.get_state().cpu().numpy(), qo, state_scale(q)) <= 1e-12
    assert s.diag()["rejected"] == 3
    s.close()


def test_inadmissible_after_max_halvings_reports_error():
    """The low-density state whose limited face pressures drive the PP wave-speed
    bound to ~1e11 cannot be stepped within 20 halvings: the step fails with
    HWENO_ERR_INADMISSIBLE and leaves the state at t^n, as the oracle reports."""
    case, q = I.random_rough(32, 32, seed=2, low=0.01)
    case.max_halvings = 20
    _, st = O.step(ocfg(case), q, dt_fixed=1e-3)
    assert st["status"] == -3
    s = hweno.Solver(case.params())
    s.set_state(torch.from_numpy(q).cuda())
    with pytest.raises(hweno.HwenoError) as e:
        s.step(1e-3)
    assert e.value.code == hweno.HWENO_ERR_INADMISSIBLE
    assert np.array_equal(s.get_state().cpu().numpy(), q)
    s.close()


def test_bitwise_determinism():
    case, q = I.random_rough(40, 36, seed=8)
    outs = []
    for _ in range(2):
        s = hweno.Solver(case.params())
        s.set_state(torch.from_numpy(q).cuda())
        s.step(1e-3)
        s.step(1e-3)
        outs.append(s.get_state().cpu().numpy())
        s.close()
    assert np.array_equal(outs[0], outs[1])


def test_host_and_device_buffers_agree():
    case, q = I.random_smooth(20, 17, seed=3)
    s = hweno.Solver(case.params())
    s.set_state(q.copy())  # host buffer
    rh = np.zeros((12, 17, 20))
    vh = np.zeros((8, 17, 20))
    s.residual(rh, vh)
    rd, vd = s.residual()
    assert np.array_equal(rh, rd.cpu().numpy()) and np.array_equal(vh, vd.cpu().numpy())
    back = np.zeros_like(q)
    s.get_state(back)
    assert np.array_equal(back, q)
    s.close()


@pytest.mark.parametrize("name", ["smooth_periodic_64", "rough_walls_45x21", "shock_tube_64x32"])
def test_mixed_precision_residual_error(name):
    """FP32 reconstruction and fluxes with FP64 state, limiter and RK: the residual
    stays within a few FP32 ulps of the FP64 oracle (relative to the plane scale)."""
    case, q = CASES[name]()
    g = gpu_residual(case, q, precision="mixed")
    o = O.residual(ocfg(case), q)
    assert rel_linf(g["rhs"], o["rhs"], flux_scale(case, q)) <= 1e-5
    assert rel_linf(g["vhat"], o["vhat"], state_scale(q)) <= 1e-6


def test_mixed_precision_conserves_to_fp64_roundoff():
    """The mixed path stores the face fluxes in FP64 and differences them in FP64, so the
    periodic cell-average residual still telescopes to FP64 round-off."""
    case, q = I.random_rough(40, 36, seed=12)
    g = gpu_residual(case, q, precision="mixed")
    for v in range(4):
        assert abs(g["rhs"][v].sum()) <= 1e-13 * np.abs(g["rhs"][v]).sum()


def test_mixed_precision_limiter_route_and_intermediates():
    """Cells the FP32 filter cannot clear take the FP64 limiter: on a low-pressure rough
    state the limited cells and theta match the FP64 path, the limited face states stay
    positive, and the FP32 intermediates stay within FP32 accuracy of the FP64 ones."""
    case, q = I.random_rough(40, 36, seed=2, low=0.01)
    gm = gpu_residual(case, q, precision="mixed", dumps=(0, 1, 2, 3, 4))
    gd = gpu_residual(case, q, precision="fp64", dumps=(0, 1, 2, 3, 4))
    lim_m = (gm[4][0] < 1) | (gm[4][1] < 1)
    lim_d = (gd[4][0] < 1) | (gd[4][1] < 1)
    assert lim_d.any() and np.array_equal(lim_m, lim_d)
    far = _far_from(lim_d, 4)
    assert rel_linf(gm[0], gd[0], state_scale(q), far) <= 1e-5
    assert rel_linf(gm[1], gd[1], state_scale(q), far) <= 1e-5
    assert rel_linf(gm["rhs"], gd["rhs"], flux_scale(case, q), far) <= 1e-5
    face = gm[0].reshape(12, 4, 36, 40)
    p = (case.gamma - 1) * (face[:, 3] - 0.5 * (face[:, 1] ** 2 + face[:, 2] ** 2) / face[:, 0])
    assert face[:, 0].min() > 0 and p.min() > 0


CONVERGENCE = {
    # a random smooth periodic field (several Fourier modes in every variable): the
    # rate is fifth order; the smooth periodic flow without its cell noise, a single density
    # wave at constant velocity and pressure, converges faster still (the leading
    # error terms cancel for it), so only at least fifth order is asked there
    "random_smooth": (lambda n: I.random_smooth(n, n, seed=31), 0.02, 4.6, 5.8),
    "smooth_periodic_wave": (lambda n: I.smooth_periodic(n, noise=0.0), 0.05, 4.6, None),
}


@pytest.mark.parametrize("name", sorted(CONVERGENCE))
def test_self_convergence_is_fifth_order(name):
    """Advance to t_end on 64^2, 128^2 and 256^2 (the viscous cap of Sec. 5 binds, so
    dt ~ h^2 and the RK3 error is O(h^6)): the differences between successive grids,
    fine solutions restricted by averaging 2x2 cells (exact for cell averages), shrink
    at the fifth-order rate in density, momentum and energy."""
    gen, t_end, lo, hi = CONVERGENCE[name]
    sols = {}
    for n in (64, 128, 256):
        case, q = gen(n)
        s = hweno.Solver(case.params())
        s.set_state(q)
        t, _ = s.advance(t_end)
        assert abs(t - t_end) < 1e-12
        sols[n] = s.get_state(np.zeros_like(q))
        s.close()

    def restrict(f):
        return 0.25 * (f[0::2, 0::2] + f[1::2, 0::2] + f[0::2, 1::2] + f[1::2, 1::2])

    for p in (0, 1, 3):
        e1 = np.abs(sols[64][p] - restrict(sols[128][p])).mean()
        e2 = np.abs(sols[128][p] - restrict(sols[256][p])).mean()
        rate = np.log2(e1 / e2)
        assert rate >= lo and (hi is None or rate <= hi), (p, e1, e2, rate)
