"""Discrete adjoint of the FP64 SSP-RK3 step: vector-Jacobian products against the
oracle's forward-mode (dual-number) tangents by dot products, against central finite
differences of the GPU forward step, the derivative with respect to mu = 1/Re, and
checkpointed or recorded multi-step rollouts (torch.autograd, record/replay).

The nonlinear weights make the step strongly curved (epsilon_WENO = 1e-8 sets the scale
of their second derivatives), so plain central differences carry an O(h^2) error with a
large constant.  The checks use Richardson-extrapolated central differences,
(4 D(h/2) - D(h)) / 3, which cancel that term."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2608_10569_b300 import hweno, inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


def richardson(f, h):
    """(4 D(h/2) - D(h)) / 3 with D(h) = (f(h) - f(-h)) / (2h)"""
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(h / 2) - f(-h / 2)) / h
    return (4 * d2 - d1) / 3


def _step(case, q, dt, Re=None):
    p = case.params()
    if Re is not None:
        p["Re"] = Re
    s = hweno.Solver(p)
    s.set_state(q.copy())
    s.step(dt)
    out = s.get_state(np.zeros_like(q))
    s.close()
    return out


CASES = {
    "periodic_smooth": lambda: I.random_smooth(20, 18, seed=31),
    "walls_smooth": lambda: I.random_smooth(19, 17, seed=32, bc=("noslip", "slip", "symmetry", "noslip")),
    "taylor_green": lambda: I.taylor_green(24, 0.5, 300.0, 1 / (1.4 * 0.09), rho_pert=1e-3),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_step_vjp_matches_central_differences(name):
    case, q = CASES[name]()
    rng = np.random.default_rng(5)
    dt = 2e-3
    lam_next = rng.normal(size=q.shape)
    v = rng.normal(size=q.shape) * np.abs(q).reshape(12, -1).max(1)[:, None, None]
    s = hweno.Solver(case.params())
    s.adjoint_init()
    lam, _ = s.adjoint_step(q.copy(), dt, lam_next, np.zeros_like(q))
    s.close()
    fd = richardson(lambda e: (_step(case, q + e * v, dt) * lam_next).sum(), 2e-6)
    ad = (lam * v).sum()
    assert abs(ad - fd) <= 1e-6 * abs(fd), (ad, fd)


def test_residual_vjp_on_a_discontinuous_state():
    """On data with jumps the weights switch between candidates and the Lax-Friedrichs
    coefficient changes hands between states, so central differences converge to the
    adjoint only as the step shrinks; the adjoint is the limit they approach."""
    case, q = I.random_rough(22, 20, seed=33)
    rng = np.random.default_rng(1)
    rb = rng.normal(size=q.shape)
    s = hweno.Solver(case.params())
    s.adjoint_init()
    xb, _ = s.adjoint_residual(q.copy(), rb, None)
    v = np.zeros_like(q)
    v[0] = rng.normal(size=q[0].shape) * np.abs(q[0]).max()
    ad = (xb * v).sum()

    def R(e):
        r = np.zeros_like(q)
        s.set_state(q + e * v)
        s.residual(r, np.zeros((8,) + q.shape[1:]))
        return (r * rb).sum()

    errs = [abs((R(h) - R(-h)) / (2 * h) - ad) / abs(ad) for h in (1e-6, 1e-7, 1e-8)]
    s.close()
    assert errs[2] < errs[1] < errs[0] and errs[2] < 2e-3, errs


def test_viscosity_derivative_matches_central_differences():
    case, q = I.random_smooth(20, 18, seed=34, Re=200.0)
    rng = np.random.default_rng(6)
    dt = 2e-3
    lam_next = rng.normal(size=q.shape)
    s = hweno.Solver(case.params())
    s.adjoint_init()
    _, mub = s.adjoint_step(q.copy(), dt, lam_next, np.zeros_like(q))
    s.close()
    mu = 1.0 / case.Re

    def diff(h):  # <lam, q(mu + h) - q(mu - h)>, the states differenced before the sum
        return (lam_next * (_step(case, q, dt, 1.0 / (mu + h)) - _step(case, q, dt, 1.0 / (mu - h)))).sum()

    h = 2e-6
    fd = (4 * diff(h / 2) / h - diff(h) / (2 * h)) / 3
    assert abs(mub - fd) <= 1e-6 * abs(fd), (mub, fd)


ORACLE_CASES = {
    "walls": lambda: I.random_smooth(16, 16, seed=35, bc=("noslip", "noslip", "noslip", "symmetry")),
    "periodic_tg": lambda: I.taylor_green(16, 0.5, 300.0, 1 / (1.4 * 0.09), rho_pert=1e-3, seed=36),
}


def _rel(a, b):
    return abs(a - b) / max(abs(a), abs(b))


@pytest.mark.parametrize("name", sorted(ORACLE_CASES))
def test_residual_vjp_dot_product_with_the_dual_oracle(name):
    """<(rbar, mbar), J (v, dmu)> from the oracle's forward-mode tangent equals
    <xbar, v> + mubar dmu from the GPU adjoint of the residual, to 1e-10"""
    case, q = ORACLE_CASES[name]()
    rng = np.random.default_rng(71)
    v = rng.normal(size=q.shape) * np.abs(q).reshape(12, -1).max(1)[:, None, None]
    rbar = rng.normal(size=q.shape)
    mbar = rng.normal(size=(8,) + q.shape[1:])
    s = hweno.Solver(case.params())
    s.adjoint_init()
    xbar, mub = s.adjoint_residual(q.copy(), rbar, mbar)
    s.close()
    cfg = O.make_cfg(**case.params())
    t = O.residual_jvp(cfg, q, v)
    tm = O.residual_jvp(cfg, q, None, dmu=1.0)
    lhs = (rbar * t["rhs_dot"]).sum() + (mbar * t["vhat_dot"]).sum()
    assert _rel(lhs, (xbar * v).sum()) <= 1e-10
    lhs_mu = (rbar * tm["rhs_dot"]).sum() + (mbar * tm["vhat_dot"]).sum()
    assert _rel(lhs_mu, mub) <= 1e-10


@pytest.mark.parametrize("name", sorted(ORACLE_CASES))
def test_step_vjp_dot_product_with_the_dual_oracle(name):
    """one SSP-RK3 step at fixed dt: <lam', J v> and <lam', dq/dmu> from the oracle's
    forward-mode tangent against <J^T lam', v> and mubar from the GPU, to 1e-10"""
    case, q = ORACLE_CASES[name]()
    rng = np.random.default_rng(72)
    dt = 1e-3
    lam_next = rng.normal(size=q.shape)
    v = rng.normal(size=q.shape) * np.abs(q).reshape(12, -1).max(1)[:, None, None]
    s = hweno.Solver(case.params())
    s.adjoint_init()
    lam, mub = s.adjoint_step(q.copy(), dt, lam_next, np.zeros_like(q))
    s.close()
    cfg = O.make_cfg(**case.params())
    _, t, st = O.step_jvp(cfg, q, v, dt)
    assert st["status"] == 0 and st["rejections"] == 0
    assert _rel((lam_next * t).sum(), (lam * v).sum()) <= 1e-10
    _, tm, _ = O.step_jvp(cfg, q, np.zeros_like(q), dt, dmu=1.0)
    assert _rel((lam_next * tm).sum(), mub) <= 1e-10


LIMITED = {
    # smooth data with eps_PP raised so that the positivity limiter acts in many cells
    # while the state stays well conditioned (at the default eps_PP = 1e-12 it acts only
    # next to vacuum, where two correct implementations agree to few digits)
    "density_factor": (37, 0.85, 0),
    "pressure_factor": (35, 0.9, 1),
}


@pytest.mark.parametrize("name", sorted(LIMITED))
def test_limiter_vjp_dot_products_with_the_dual_oracle(name):
    """residual and step adjoints where the limiter acts, against the oracle's
    forward-mode tangents, to 1e-10"""
    seed, eps_pp, which = LIMITED[name]
    case, q = I.random_smooth(16, 16, seed=seed, bc=("noslip", "noslip", "noslip", "symmetry"))
    p = case.params()
    p["eps_pp"] = eps_pp
    cfg = O.make_cfg(**p)
    th = O.residual(cfg, q, dumps=True)["theta"]
    assert (th[which] < 1).sum() >= 5
    rng = np.random.default_rng(74)
    v = rng.normal(size=q.shape) * np.abs(q).reshape(12, -1).max(1)[:, None, None]
    rbar = rng.normal(size=q.shape)
    mbar = rng.normal(size=(8,) + q.shape[1:])
    s = hweno.Solver(p)
    s.adjoint_init()
    xbar, mub = s.adjoint_residual(q.copy(), rbar, mbar)
    t = O.residual_jvp(cfg, q, v)
    tm = O.residual_jvp(cfg, q, None, dmu=1.0)
    assert _rel((rbar * t["rhs_dot"]).sum() + (mbar * t["vhat_dot"]).sum(), (xbar * v).sum()) <= 1e-10
    assert _rel((rbar * tm["rhs_dot"]).sum() + (mbar * tm["vhat_dot"]).sum(), mub) <= 1e-10
    dt = 0.25 * O.step(cfg, q)[1]["dt"]
    lam_next = rng.normal(size=q.shape)
    lam, mub = s.adjoint_step(q.copy(), dt, lam_next, np.zeros_like(q))
    s.close()
    _, ts, st = O.step_jvp(cfg, q, v, dt)
    assert st["status"] == 0 and st["rejections"] == 0 and st["pp_active"] > 0
    assert _rel((lam_next * ts).sum(), (lam * v).sum()) <= 1e-10
    _, tms, _ = O.step_jvp(cfg, q, np.zeros_like(q), dt, dmu=1.0)
    assert _rel((lam_next * tms).sum(), mub) <= 1e-10


def test_adjoint_taylor_green_replica_dot_product_with_the_dual_oracle():
    """the adjoint Taylor-Green flow (Re 1600, Mach 0.3) on a 64^2 replica: three
    recorded steps under the step rule against the oracle's forward-mode tangent, for
    the initial state and for mu, to 1e-10 or ten times the products' own sensitivity
    to rounding-level changes of the state, whichever is larger"""
    case, q = I.adjoint_taylor_green(64)
    rng = np.random.default_rng(75)
    lam_T = rng.normal(size=q.shape)
    v = rng.normal(size=q.shape) * np.abs(q).reshape(12, -1).max(1)[:, None, None]
    s = hweno.Solver(case.params())
    s.set_state(q.copy())
    s.adjoint_init()
    s.adjoint_reserve(3)
    s.adjoint_record(True)
    dts = [s.step()[0] for _ in range(3)]
    lam0, mub = s.adjoint_replay(lam_T.copy(), np.zeros_like(q))
    s.close()
    cfg = O.make_cfg(**case.params())

    def tangents(q0):
        qa, ta, qb, tb = q0.copy(), v.copy(), q0.copy(), np.zeros_like(q0)
        for dt in dts:
            qa, ta, _ = O.step_jvp(cfg, qa, ta, dt)
            qb, tb, _ = O.step_jvp(cfg, qb, tb, dt, dmu=1.0)
        return (lam_T * ta).sum(), (lam_T * tb).sum()

    ref_q, ref_mu = tangents(q)
    # conditioning: how far the oracle's own products move when the state moves by
    # rounding (2e-16 relative), as the GPU's forward states differ from the oracle's.
    # The replica's density starts uniform, so smoothness indicators sit near eps_WENO
    # and the weights' second derivatives amplify rounding to about 1e-9.
    sens_q, sens_mu = 0.0, 0.0
    for k in range(2):
        pq, pmu = tangents(q * (1.0 + 2e-16 * np.random.default_rng(200 + k).normal(size=q.shape)))
        sens_q, sens_mu = max(sens_q, _rel(pq, ref_q)), max(sens_mu, _rel(pmu, ref_mu))
    assert _rel(ref_q, (lam0 * v).sum()) <= max(1e-10, 10 * sens_q)
    assert _rel(ref_mu, mub) <= max(1e-10, 10 * sens_mu)


def test_recorded_rollout_dot_product_with_the_dual_oracle():
    """five recorded steps under the step rule, reversed by hweno_adjoint_replay, against
    the oracle's tangent through the same five steps (the GPU's step sizes), to 1e-10"""
    case, q = ORACLE_CASES["walls"]()
    rng = np.random.default_rng(73)
    lam_T = rng.normal(size=q.shape)
    v = rng.normal(size=q.shape) * np.abs(q).reshape(12, -1).max(1)[:, None, None]
    s = hweno.Solver(case.params())
    s.set_state(q.copy())
    s.adjoint_init()
    s.adjoint_reserve(5)
    s.adjoint_record(True)
    dts = [s.step()[0] for _ in range(5)]
    s.adjoint_record(False)
    lam0, mub = s.adjoint_replay(lam_T.copy(), np.zeros_like(q))
    s.close()
    cfg = O.make_cfg(**case.params())
    qa, ta, qb, tb = q.copy(), v.copy(), q.copy(), np.zeros_like(q)
    for dt in dts:
        qa, ta, _ = O.step_jvp(cfg, qa, ta, dt)
        qb, tb, _ = O.step_jvp(cfg, qb, tb, dt, dmu=1.0)
    assert _rel((lam_T * ta).sum(), (lam0 * v).sum()) <= 1e-10
    assert _rel((lam_T * tb).sum(), mub) <= 1e-10


def test_checkpointed_rollout_gradient():
    """J = 1/2 sum (rho(T) - rho*)^2 dx dy over 12 steps with checkpoints every 5 steps:
    dJ/dq0 and dJ/dmu through torch.autograd against central differences on random
    directions (the step sizes recorded in the forward are reused)."""
    case, q = I.taylor_green(24, 0.5, 400.0, 1 / (1.4 * 0.09), rho_pert=1e-3, seed=8)
    params = case.params()
    q0 = torch.from_numpy(q).cuda().requires_grad_(True)
    mu = torch.tensor(1.0 / case.Re, dtype=torch.float64, device="cuda", requires_grad=True)
    rng = np.random.default_rng(9)
    target = torch.from_numpy(q[0] + 1e-2 * rng.normal(size=q[0].shape)).cuda()
    area = case.dx * case.dy

    def J(qT):
        return 0.5 * ((qT[0] - target) ** 2).sum() * area

    qT = hweno.rollout(q0, mu, params, nsteps=12, ckpt=5)
    loss = J(qT)
    loss.backward()
    g0 = q0.grad.cpu().numpy()
    gmu = float(mu.grad)
    # replay with the same step sizes for the differences
    s = hweno.Solver(params)
    s.set_state(q.copy())
    dts = [s.step()[0] for _ in range(12)]
    s.close()

    def run(qi, Re):
        p = dict(params)
        p["Re"] = Re
        s = hweno.Solver(p)
        s.set_state(qi.copy())
        for dt in dts:
            s.step(dt)
        out = s.get_state(np.zeros_like(qi))
        s.close()
        return float(J(torch.from_numpy(out).cuda()))

    scale = np.abs(q).reshape(12, -1).max(1)[:, None, None]
    for k in range(3):
        v = rng.normal(size=q.shape) * scale
        fd = richardson(lambda e: run(q + e * v, case.Re), 1e-7)
        assert abs((g0 * v).sum() - fd) <= 1e-6 * abs(fd), ((g0 * v).sum(), fd)
    mu0 = 1.0 / case.Re
    fdmu = richardson(lambda e: run(q, 1.0 / (mu0 + e)), 2e-6)
    assert abs(gmu - fdmu) <= 1e-6 * abs(fdmu), (gmu, fdmu)


@pytest.mark.parametrize("keep", [True, False])
def test_segment_adjoint_equals_chained_steps(keep):
    """hweno_adjoint_segment (one forward recomputation, stored stage states, with or
    without stored intermediates) equals the chain of single-step adjoints."""
    case, q = I.taylor_green(20, 0.4, 300.0, 1 / (1.4 * 0.09), rho_pert=1e-3, seed=10)
    rng = np.random.default_rng(11)
    lam_end = rng.normal(size=q.shape)
    s = hweno.Solver(case.params())
    s.set_state(q.copy())
    states, dts = [q.copy()], []
    for _ in range(4):
        dts.append(s.step()[0])
        states.append(s.get_state(np.zeros_like(q)))
    s.adjoint_init()
    lam, mub = lam_end.copy(), 0.0
    for k in range(3, -1, -1):
        lam, mb = s.adjoint_step(states[k].copy(), dts[k], lam, np.zeros_like(q))
        mub += mb
    kept = s.adjoint_reserve(4, keep_intermediates=keep)
    assert kept == keep
    lam2, mub2 = s.adjoint_segment(q.copy(), dts, lam_end.copy(), np.zeros_like(q))
    s.close()
    assert np.abs(lam2 - lam).max() <= 1e-12 * np.abs(lam).max()
    assert abs(mub2 - mub) <= 1e-12 * abs(mub)


@pytest.mark.parametrize("keep", [True, False])
def test_recorded_steps_replay_equals_chained_steps(keep):
    """Steps recorded while hweno_step runs (hweno_adjoint_record), reversed by
    hweno_adjoint_replay, give the chain of single-step adjoints at the recorded step
    sizes; the replay leaves the solver's state alone, and recording more steps than
    reserved is an error."""
    case, q = I.taylor_green(20, 0.4, 300.0, 1 / (1.4 * 0.09), rho_pert=1e-3, seed=12)
    rng = np.random.default_rng(13)
    lam_end = rng.normal(size=q.shape)
    s = hweno.Solver(case.params())
    s.set_state(q.copy())
    s.adjoint_init()
    assert s.adjoint_reserve(3, keep_intermediates=keep) == keep
    s.step()  # not recorded
    states = [s.get_state(np.zeros_like(q))]
    s.adjoint_record(True)
    dts = []
    for _ in range(3):
        dts.append(s.step()[0])
        states.append(s.get_state(np.zeros_like(q)))
    s.adjoint_record(False)
    s.step()  # not recorded either
    q_after = s.get_state(np.zeros_like(q))
    lam, mub = s.adjoint_replay(lam_end.copy(), np.zeros_like(q))
    assert np.array_equal(s.get_state(np.zeros_like(q)), q_after)
    lam2, mub2 = lam_end.copy(), 0.0
    for k in range(2, -1, -1):
        lam2, mb = s.adjoint_step(states[k].copy(), dts[k], lam2, np.zeros_like(q))
        mub2 += mb
    assert np.abs(lam - lam2).max() <= 1e-12 * np.abs(lam2).max()
    assert abs(mub - mub2) <= 1e-12 * abs(mub2)
    s.set_state(q.copy())
    s.adjoint_record(True)
    for _ in range(3):
        s.step()
    with pytest.raises(hweno.HwenoError, match="reserve"):
        s.step()
    s.close()
