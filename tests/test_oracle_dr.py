"""Pins of the oracle's HWENO-DR gradients (the paper's comparison scheme, Eq. (3.5)):
the derivatives of the characteristic candidate polynomials, combined with the nonlinear
weights of the convective reconstruction, replace the weak-derivative reconstruction of
Eq. (3.9).

What fixes them independently of the oracle:
  * exact polynomial derivatives (numpy's polyder; sympy for the rational (u, v, e)
    fields) where the linear weights reduce the combination to p0;
  * the divergence theorem on the reference cell, which ties the derivatives of the
    nonlinear combination, for any data, to the already pinned value reconstruction
    (face values and the preserved cell average);
  * the Euler limit, where the viscous gradients drop out and DR and GR coincide;
  * the orders the paper states: fourth for DR, fifth for GR (Sec. 3.1, Table 5.2).
"""
import math

import numpy as np
import pytest
import sympy as sp
from numpy.polynomial import polynomial as npoly

from oracle import oracle as O
from paper_2608_10569_b300 import inputs as I
from test_oracle_pins import (FACE_PTS, MONOS, VOL_PTS, _cfg, _manufactured, _mirror_x, _moments_of,
                              _transpose)

GW = np.array([5 / 18, 4 / 9, 5 / 18])
GN = np.array([-1.0, 0.0, 1.0]) * math.sqrt(15.0) / 10.0


def _grid_of(c):
    """monomial coefficients (order of MONOS) -> numpy 2D coefficient grid [p][q]"""
    C = np.zeros((5, 5))
    for k, (p, q) in enumerate(MONOS):
        C[p, q] = c[k]
    return C


# ---------------------------------------------------------------------------
# one scalar reconstruction

@pytest.mark.parametrize("seed", range(3))
def test_scalar_derivatives_exact_for_quartics_with_linear_weights(seed):
    """omega = gamma turns the DR combination into p0', and p0 is the data's quartic
    (Appendix A.2), so the derivatives are the polynomial's own at all 21 points."""
    c = np.random.default_rng(10 + seed).normal(size=15)
    C = _grid_of(c)
    d, _, _ = _moments_of(lambda x, y: npoly.polyval2d(x, y, C))
    dxi, deta = O.hweno_scalar_dr(d, linear=True)
    pts = np.array(FACE_PTS + VOL_PTS)
    ex = npoly.polyval2d(pts[:, 0], pts[:, 1], npoly.polyder(C, axis=0))
    ey = npoly.polyval2d(pts[:, 0], pts[:, 1], npoly.polyder(C, axis=1))
    assert np.abs(dxi - ex).max() < 1e-11
    assert np.abs(deta - ey).max() < 1e-11


def test_scalar_derivatives_of_a_linear_field_for_any_weights():
    """all five candidates of linear data are that plane and the weights sum to one,
    so every point returns its slope, whatever the nonlinear weights"""
    d, _, _ = _moments_of(lambda x, y: 0.3 + 1.7 * x - 0.4 * y)
    for eps in (1e-8, 1e-2):
        dxi, deta = O.hweno_scalar_dr(d, eps=eps)
        assert np.abs(dxi - 1.7).max() < 1e-13 and np.abs(deta + 0.4).max() < 1e-13


@pytest.mark.parametrize("seed", range(4))
def test_divergence_theorem_ties_derivatives_to_the_values(seed):
    """The weights are constant over the cell, so the DR derivatives are those of the
    reconstructed value polynomial u (a quartic).  On the cell [-1/2, 1/2]^2 the
    divergence theorem gives, with 3-point Gauss exact for every integrand here
    (degree <= 5 per variable):
        sum_GH w_G w_H u_xi(xi_G, eta_H)       = sum_H w_H (u(1/2, eta_H) - u(-1/2, eta_H))
        sum_GH w_G w_H xi_G u_xi(xi_G, eta_H)  = sum_H w_H (u(1/2, eta_H) + u(-1/2, eta_H))/2 - ubar
        sum_GH w_G w_H eta_H u_xi(xi_G, eta_H) = sum_H w_H eta_H (u(1/2, eta_H) - u(-1/2, eta_H))
    and the same with the roles of xi and eta exchanged.  The values u come from the
    pinned value reconstruction and ubar is the centre average it preserves; random data
    make the nonlinear weights differ from the linear ones."""
    rng = np.random.default_rng(20 + seed)
    d = rng.normal(size=17) * rng.uniform(0.5, 5.0)
    o = O.hweno_scalar(d)
    assert np.abs(o["omega"] - np.array([0.99] + [0.0025] * 4)).max() > 1e-3
    dxi, deta = O.hweno_scalar_dr(d)
    pts = o["pts"]
    left, right, bottom, top = pts[0:3], pts[3:6], pts[6:9], pts[9:12]
    W2 = np.outer(GW, GW)
    DX = dxi[12:].reshape(3, 3)   # [G][H] at (xi_G, eta_H)
    DY = deta[12:].reshape(3, 3)
    XI = np.outer(GN, np.ones(3))
    ETA = np.outer(np.ones(3), GN)
    scale = max(1.0, np.abs(d).max())
    tol = 1e-12 * scale
    assert abs((W2 * DX).sum() - GW @ (right - left)) < tol
    assert abs((W2 * XI * DX).sum() - (0.5 * GW @ (right + left) - d[4])) < tol
    assert abs((W2 * ETA * DX).sum() - GW @ (GN * (right - left))) < tol
    assert abs((W2 * DY).sum() - GW @ (top - bottom)) < tol
    assert abs((W2 * ETA * DY).sum() - (0.5 * GW @ (top + bottom) - d[4])) < tol
    assert abs((W2 * XI * DY).sum() - GW @ (GN * (top - bottom))) < tol


# ---------------------------------------------------------------------------
# whole spatial operator

def _quartic_conserved_case(n, gamma=1.4):
    """quartic conserved fields with a varying density on [0,1]^2, as sympy
    expressions and as cell moments"""
    x, y = sp.symbols("x y")
    rho = 1.5 + sp.Rational(1, 5) * x ** 2 - sp.Rational(1, 10) * x * y + sp.Rational(1, 20) * y ** 3
    m = sp.Rational(1, 2) + x ** 2 - sp.Rational(3, 10) * x * y + sp.Rational(1, 10) * y ** 4
    nn = -sp.Rational(1, 5) + y ** 2 + sp.Rational(1, 10) * x - sp.Rational(2, 5) * x ** 3 * y
    E = 4 + x ** 4 + sp.Rational(1, 2) * x * y ** 3 - sp.Rational(7, 10) * x * x * y
    f = [sp.lambdify((x, y), e, "numpy") for e in (rho, m, nn, E)]
    case = I.Case("quartic", n, n, gamma=gamma, Re=100.0)

    def prim(X, Y):
        r, mm, n2, e = (np.broadcast_to(fi(X, Y), np.shape(X)).astype(float) for fi in f)
        return r, mm / r, n2 / r, (gamma - 1) * (e - 0.5 * (mm * mm + n2 * n2) / r)

    q = I.cell_moments(case, prim, nq=6)
    u, v = m / rho, nn / rho
    e = E / rho - (u * u + v * v) / 2
    grads = [sp.diff(w, s) for w in (u, v, e) for s in (x, y)]
    g = sp.lambdify((x, y), grads, "numpy")
    return case, q, g


def test_gradients_exact_for_quartic_conserved_fields():
    """Linear weights, no limiter: each characteristic field is a quartic that p0
    recovers, so both systems' derivatives are exact, and the chain rule to
    (u, v, e) returns the exact rational gradients at all 21 points of every cell
    whose stencil avoids the periodic seam."""
    n = 16
    h = 1.0 / n
    case, q, g = _quartic_conserved_case(n)
    r = O.residual(_cfg(case, linear_weights=True, limiter=False, scheme="dr"), q, dumps=True)
    worst = 0.0
    for j in range(4, n - 4):
        for i in range(4, n - 4):
            xc, yc = (i + 0.5) * h, (j + 0.5) * h
            for k, (a, b) in enumerate(FACE_PTS + VOL_PTS):
                ex = np.array(g(xc + a * h, yc + b * h), dtype=float)
                worst = max(worst, np.abs(r["grad"][6 * k:6 * k + 6, j, i] - ex).max())
    assert worst < 1e-9, worst


def _gradient_errors(n, scheme, linear=False):
    """max and mean point-gradient errors over the 21 points of every cell"""
    gamma, Pr, Re = 1.4, 0.72, 100.0
    h = 1.0 / n
    case = I.Case("mms", n, n, gamma=gamma, Pr=Pr, Re=Re)

    def prim(x, y):
        rho, u, v, e, _ = _manufactured(x, y)
        return rho, u, v, (gamma - 1) * rho * e

    q = I.cell_moments(case, prim, nq=6)
    r = O.residual(_cfg(case, scheme=scheme, linear_weights=linear), q, dumps=True)
    xc = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(xc, xc)
    emax, esum = 0.0, 0.0
    for k, (a, b) in enumerate(FACE_PTS + VOL_PTS):
        ex = _manufactured(X + a * h, Y + b * h)[4]
        for c6 in range(6):
            d = np.abs(r["grad"][6 * k + c6] - ex[c6])
            emax = max(emax, d.max())
            esum += d.sum()
    return np.array([emax, esum / (126 * n * n)])


@pytest.mark.parametrize("linear", [True, False], ids=["linear_weights", "nonlinear_weights"])
def test_dr_gradients_are_fourth_order_and_gr_fifth(linear):
    """Sec. 3.1: differentiating the fifth-order reconstruction loses one order; the
    weak-derivative reconstruction of Sec. 3.2 keeps the fifth (Table 5.2's DR and GR
    rows).  Point-gradient errors (max and mean) on Example 5.2's fields.  With the
    nonlinear weights both schemes pass through a transient of higher apparent rates on
    coarse meshes while the weights approach the linear ones, as Table 5.2's DR rows
    do; 96 -> 192 is past it."""
    ns = (48, 96) if linear else (96, 192)
    dr = [_gradient_errors(n, "dr", linear) for n in ns]
    gr = [_gradient_errors(n, "gr", linear) for n in ns]
    rate_dr = np.log2(dr[0] / dr[1])
    rate_gr = np.log2(gr[0] / gr[1])
    assert np.all((rate_dr > 3.8) & (rate_dr < 4.2)), (dr, rate_dr)
    assert np.all(rate_gr > 4.8), (gr, rate_gr)
    assert dr[1][0] > 10 * gr[1][0]


@pytest.mark.parametrize("kind", ["smooth", "rough"])
def test_euler_limit_dr_equals_gr(kind):
    """Sec. 5: the two schemes share the convective discretisation, so with 1/Re = 0
    (no viscous flux) their residuals agree to the bit; at finite Re they differ."""
    bc = ("noslip", "symmetry", "slip", "noslip")
    mk = I.random_smooth if kind == "smooth" else I.random_rough
    case, q = mk(14, 12, seed=8, bc=bc)
    r_gr = O.residual(_cfg(case, Re=math.inf), q)
    r_dr = O.residual(_cfg(case, Re=math.inf, scheme="dr"), q)
    assert np.array_equal(r_gr["rhs"], r_dr["rhs"])
    assert np.array_equal(r_gr["vhat"], r_dr["vhat"])
    v_gr = O.residual(_cfg(case), q)["rhs"]
    v_dr = O.residual(_cfg(case, scheme="dr"), q)["rhs"]
    assert np.abs(v_gr - v_dr).max() > 1e-8 * np.abs(v_gr).max()


def test_free_stream_and_conservation():
    """P2/P3 under DR: a constant state has zero residual; on a periodic grid the
    cell-average residual sums to zero."""
    case = I.Case("fs", 12, 10, Re=50.0)
    q = np.zeros((12, 10, 12))
    U = I.conserved(1.3, 0.4, -0.2, 2.0, 1.4)
    for k in range(4):
        q[k] = U[k]
    r = O.residual(_cfg(case, scheme="dr"), q, dumps=True)
    assert np.abs(r["rhs"]).max() < 1e-13 and np.abs(r["grad"]).max() < 1e-13
    for mk in (I.random_smooth, I.random_rough):
        case, q = mk(20, 16, seed=2)
        rhs = O.residual(_cfg(case, scheme="dr"), q)["rhs"]
        for v in range(4):
            assert abs(rhs[v].sum()) < 1e-13 * max(np.abs(rhs[v]).sum(), 1.0)


@pytest.mark.parametrize("kind", ["smooth", "rough"])
def test_transpose_and_mirror_equivariance(kind):
    """P5 under DR: x<->y and x -> -x commute with the residual, so each system
    differentiates at its own faces and the volume points treat the systems alike."""
    bc = ("noslip", "symmetry", "slip", "noslip")
    mk = I.random_smooth if kind == "smooth" else I.random_rough
    case, q = mk(14, 11, seed=4, bc=bc)
    r1 = O.residual(_cfg(case, scheme="dr"), q)
    case_t = I.Case("t", case.ny, case.nx, case.y0, case.y1, case.x0, case.x1, case.gamma, case.Pr,
                    case.Re, bc=(bc[2], bc[3], bc[0], bc[1]))
    r2 = O.residual(_cfg(case_t, scheme="dr"), _transpose(q, 12))
    a, b = _transpose(r1["rhs"], 12), r2["rhs"]
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    bc = ("noslip", "symmetry", "periodic", "periodic")
    case, q = mk(13, 10, seed=5, bc=bc)
    r1 = O.residual(_cfg(case, scheme="dr"), q)
    case_m = I.Case("m", case.nx, case.ny, case.x0, case.x1, case.y0, case.y1, case.gamma, case.Pr,
                    case.Re, bc=(bc[1], bc[0], bc[2], bc[3]))
    r2 = O.residual(_cfg(case_m, scheme="dr"), _mirror_x(q))
    a, b = _mirror_x(r1["rhs"]), r2["rhs"]
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_limiter_enters_only_through_the_limited_traces():
    """The limiter leaves the derivatives alone; the chain rule to (u, v, e) takes the
    state the fluxes use at each point.  On colliding near-vacuum streams (limiter
    engaged) the DR residual stays finite; against the run without limiter, the volume
    gradients (volume values are never limited) agree to the bit, the face gradients of
    cells the limiter left alone to rounding (the limiter rewrites every face value as
    ubar + theta (u - ubar), also with theta = 1), and those of the limited cells
    change."""
    case, q = I.colliding_streams(32, seed=3)
    on = O.residual(_cfg(case, scheme="dr"), q, dumps=True)
    off = O.residual(_cfg(case, scheme="dr", limiter=False), q, dumps=True)
    limited = (on["theta"][0] < 1) | (on["theta"][1] < 1)
    assert limited.any() and (~limited).any()
    assert np.isfinite(on["rhs"]).all()
    assert np.array_equal(on["grad"][72:], off["grad"][72:])
    a, b = on["grad"][:72, ~limited], off["grad"][:72, ~limited]
    scale = np.abs(b).max(axis=1, keepdims=True)
    assert (np.abs(a - b) <= 1e-10 * scale).all()
    a, b = on["grad"][:72, limited], off["grad"][:72, limited]
    assert np.abs(a - b).max() > 1e-3 * np.abs(b).max()
