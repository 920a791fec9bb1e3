"""Pins of the oracle's manufactured source (Example 5.2): S = U_t + F_x + G_y for the
manufactured fields, its cell moments, and its stage times in the SSP-RK3 step.

Independent facts: sympy differentiates the conserved variables and the full fluxes
symbolically; the exact time derivative of the manufactured solution is known in closed
form (every perturbation decays like exp(-t)); SSP-RK3 samples a time-dependent
right-hand side at the nodes of its Butcher tableau; and the error of a run against the
exact solution must fall at the scheme's spatial order once the time step scales like
h^2.
"""
import math

import numpy as np
import pytest
import sympy as sp

from oracle import oracle as O
from paper_2608_10569_b300 import inputs as I


def _symbolic_source(gamma, Pr, Re):
    x, y, t = sp.symbols("x y t")
    a = sp.Rational(1, 10) * sp.exp(-t)
    tp = 2 * sp.pi
    rho = 2 + a * (sp.sin(tp * (2 * x - y)) + sp.cos(tp * (-x + 2 * y)))
    u = 1 + a * (sp.sin(tp * (-x + y)) + sp.cos(tp * (x + y)))
    v = 2 + a * (sp.sin(tp * (x + y)) + sp.cos(tp * (x - y)))
    e = 2 + a * (sp.sin(tp * (x - y)) + sp.cos(tp * (x + y)))
    p = (gamma - 1) * rho * e
    E = rho * (e + (u * u + v * v) / 2)
    txx = sp.Rational(4, 3) * sp.diff(u, x) - sp.Rational(2, 3) * sp.diff(v, y)
    tyy = sp.Rational(4, 3) * sp.diff(v, y) - sp.Rational(2, 3) * sp.diff(u, x)
    txy = sp.diff(u, y) + sp.diff(v, x)
    U = [rho, rho * u, rho * v, E]
    F = [rho * u, rho * u * u + p - txx / Re, rho * u * v - txy / Re,
         u * (E + p) - (txx * u + txy * v + gamma / Pr * sp.diff(e, x)) / Re]
    G = [rho * v, rho * u * v - txy / Re, rho * v * v + p - tyy / Re,
         v * (E + p) - (txy * u + tyy * v + gamma / Pr * sp.diff(e, y)) / Re]
    S = [sp.diff(U[k], t) + sp.diff(F[k], x) + sp.diff(G[k], y) for k in range(4)]
    return sp.lambdify((x, y, t), S, "numpy")


@pytest.mark.parametrize("Re", [100.0, 7.0])
def test_source_matches_symbolic_differentiation(Re):
    """the oracle's hand-differentiated S equals sympy's derivative of the conserved
    variables and fluxes of Example 5.2's equations"""
    f = _symbolic_source(1.4, 0.72, Re)
    cfg = O.make_cfg(8, 8, Re=Re, source=1)
    rng = np.random.default_rng(52)
    for _ in range(24):
        x, y = rng.uniform(0, 1, 2)
        t = rng.choice([0.0, 0.05, 0.3])
        ex = np.array(f(x, y, t), dtype=float)
        got = O.mms_source(cfg, x, y, t)
        assert np.abs(got - ex).max() <= 1e-12 * np.abs(ex).max(), (x, y, t, got, ex)


def _exact_ut_moments(case, t):
    """cell moments of U_t for the manufactured solution: each perturbation decays like
    exp(-t), so rho_t = -(rho - 2), u_t = -(u - 1), v_t = -(v - 2), e_t = -(e - 2)"""
    g = case.gamma
    gn, gw = np.polynomial.legendre.leggauss(6)
    gn, gw = 0.5 * gn, 0.5 * gw
    n = case.nx
    h = 1.0 / n
    xc = (np.arange(n) + 0.5) * h
    out = np.zeros((12, n, n))
    for a in range(len(gn)):
        for b in range(len(gn)):
            X, Y = np.broadcast_arrays((xc + gn[a] * h)[None, :], (xc + gn[b] * h)[:, None])
            rho, u, v, p = I.manufactured_prim(X, Y, t, g)
            e = p / ((g - 1) * rho)
            rt, ut, vt, et = -(rho - 2), -(u - 1), -(v - 2), -(e - 2)
            k = 0.5 * (u * u + v * v)
            Ut = [rt, rt * u + rho * ut, rt * v + rho * vt, rt * (e + k) + rho * (et + u * ut + v * vt)]
            w = gw[a] * gw[b]
            for c in range(4):
                out[c] += w * Ut[c]
                out[4 + c] += w * gn[a] * Ut[c]
                out[8 + c] += w * gn[b] * Ut[c]
    return out


def test_semi_discrete_system_is_consistent():
    """R(U) + S-bar against the exact d/dt of the cell moments of the manufactured
    solution at t = 0.05 (linear weights, so that the rates are asymptotic on these
    meshes): the averages converge at the scheme's fifth order (Sec. 3.2), the scaled
    first moments at fourth; a wrong source term or source moment would leave an O(1)
    error"""
    t = 0.05
    errs = []
    for n in (48, 96):
        case, q = I.manufactured(n, t)
        r = O.residual(O.make_cfg(**case.params(), time=t, linear_weights=True), q)["rhs"]
        d = np.abs(r - _exact_ut_moments(case, t))
        errs.append([d[4 * m:4 * m + 4].max() for m in range(3)])
    rates = [math.log2(errs[0][m] / errs[1][m]) for m in range(3)]
    assert 4.8 < rates[0] < 5.3, (errs, rates)
    assert rates[1] > 3.8 and rates[2] > 3.8, (errs, rates)
    assert errs[1][0] < 1e-5


def test_step_matches_butcher_form_with_stage_times():
    """A non-autonomous right-hand side dU/dt = R(U) + S(t) is sampled by SSP-RK3 at the
    nodes of its Butcher tableau, c = A 1 = (0, 1, 1/2) for a21 = 1, a31 = a32 = 1/4.
    The oracle's Shu-Osher step (Eq. (2.12)) with the source equals the Butcher form
    evaluated at t0 + c dt, with each stage's first moments taken as Eq. (2.12) states
    (modified moment of the stage plus dt times the moment residual)."""
    case, q = I.manufactured(16, 0.02)
    t0, dt = 0.02, 4e-3
    A = np.array([[0, 0, 0], [1, 0, 0], [0.25, 0.25, 0]])
    c = A.sum(axis=1)

    def F(y, k):
        r = O.residual(O.make_cfg(**case.params(), time=t0 + c[k] * dt), y)
        return r["rhs"], r["vhat"]

    k1, vh0 = F(q, 0)
    y1 = np.concatenate([q[:4] + dt * k1[:4], vh0 + dt * k1[4:]])
    k2, vh1 = F(y1, 1)
    y2 = np.concatenate([q[:4] + dt / 4 * (k1[:4] + k2[:4]), 0.75 * vh0 + 0.25 * (vh1 + dt * k2[4:])])
    k3, vh2 = F(y2, 2)
    avg = q[:4] + dt / 6 * (k1[:4] + k2[:4] + 4 * k3[:4])
    mom = vh0 / 3 + 2 / 3 * (vh2 + dt * k3[4:])
    q1, st = O.step(O.make_cfg(**case.params()), q, t=t0, dt_fixed=dt)
    assert st["dt"] == dt and st["rejections"] == 0
    assert np.abs(q1[:4] - avg).max() < 1e-13 * np.abs(avg).max()
    assert np.abs(q1[4:] - mom).max() < 1e-13 * np.abs(mom).max()


def test_time_convergence_with_source():
    """Runs to T = 0.01 under the Sec. 5 step rule (dt = b Re h^2 here, so the time error
    O(dt^3) = O(h^6) is below the spatial one): the density error against the exact
    solution falls at about the fifth order"""
    errs = []
    for n in (16, 32):
        case, q = I.manufactured(n, 0.0)
        qT, st = O.advance(O.make_cfg(**case.params()), q, 0.0, 0.01)
        assert st["status"] == 0
        _, qex = I.manufactured(n, 0.01)
        errs.append(np.abs(qT[0] - qex[0]).mean())
    rate = math.log2(errs[0] / errs[1])
    assert rate > 4.4, (errs, rate)


def test_source_tangent_in_mu():
    """the dual build differentiates the source too (it depends on mu = 1/Re): the
    residual's mu-tangent with the source on equals Richardson differences"""
    case, q = I.manufactured(12, 0.02)
    p = dict(case.params(), time=0.02)
    mu0 = 1.0 / case.Re
    tm = O.residual_jvp(O.make_cfg(**p), q, None, dmu=1.0)["rhs_dot"]

    def at(e):
        pp = dict(p)
        pp["Re"] = 1.0 / (mu0 + e)
        return O.residual(O.make_cfg(**pp), q)["rhs"]

    h = 1e-2 * mu0
    fd = (4 * (at(h / 2) - at(-h / 2)) / h - (at(h) - at(-h)) / (2 * h)) / 3
    assert np.abs(tm - fd).max() <= 1e-8 * np.abs(tm).max()
