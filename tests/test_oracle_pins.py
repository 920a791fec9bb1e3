"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks a property that an independent fact determines (exact
polynomial recovery, free stream, conservation, positivity, symmetry, order of
accuracy, an equivalent RK form, a brute-force root), so that a dropped term, a wrong
sign or index, or a transposed operand in the oracle fails one of them.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_10569_b300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
G = math.sqrt(15.0) / 10.0
MONOS = [(p, d - p) for d in range(5) for p in range(d, -1, -1)]
FACE_PTS = ([(-0.5, -G), (-0.5, 0.0), (-0.5, G), (0.5, -G), (0.5, 0.0), (0.5, G),
             (-G, -0.5), (0.0, -0.5), (G, -0.5), (-G, 0.5), (0.0, 0.5), (G, 0.5)])
VOL_PTS = [(a, b) for a in (-G, 0.0, G) for b in (-G, 0.0, G)]


def golden_constants():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_constants.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, val = line.split()[:2]
            out[name] = float(val)
    return out


# ---------------------------------------------------------------------------
# scalar reconstruction (Appendix A.2)

def _moments_of(P, nq=6):
    """the 17 data of the 3x3 stencil for a point function P(xi, eta) in the
    centre cell's scaled coordinates (high-order Gauss, exact for the quartics used)"""
    gn, gw = np.polynomial.legendre.leggauss(nq)
    gn, gw = 0.5 * gn, 0.5 * gw

    def m(a, b, wx=0, wy=0):
        s = 0.0
        for i in range(nq):
            for j in range(nq):
                s += gw[i] * gw[j] * P(a + gn[i], b + gn[j]) * (gn[i] if wx else 1) * (gn[j] if wy else 1)
        return s

    lab = {k + 1: ((k % 3) - 1, (k // 3) - 1) for k in range(9)}
    d = [m(*lab[k]) for k in range(1, 10)]
    d += [m(*lab[4], wx=1), m(*lab[6], wx=1), m(*lab[2], wy=1), m(*lab[8], wy=1),
          m(*lab[2], wx=1), m(*lab[8], wx=1), m(*lab[4], wy=1), m(*lab[6], wy=1)]
    return np.array(d), m(0, 0, wx=1), m(0, 0, wy=1)


@pytest.mark.parametrize("seed", range(4))
def test_quartic_recovered_exactly_with_linear_weights(seed):
    """P1: any polynomial of degree <= 4 satisfies all 17 conditions exactly, so the
    constrained least-squares quartic is that polynomial (Appendix A.2, Eq. (A.4));
    with omega = gamma the combination of Eq. (3.4) returns p0."""
    c = np.random.default_rng(seed).normal(size=15)

    def P(x, y):
        return sum(c[k] * x ** MONOS[k][0] * y ** MONOS[k][1] for k in range(15))

    d, mx, my = _moments_of(P)
    o = O.hweno_scalar(d, linear=True)
    assert np.abs(o["c0"] - c).max() < 1e-12
    exact = np.array([P(*p) for p in FACE_PTS + VOL_PTS])
    assert np.abs(o["pts"] - exact).max() < 1e-12
    assert abs(o["mom"][0] - mx) < 1e-13 and abs(o["mom"][1] - my) < 1e-13


def test_constrained_least_squares_matches_numeric_kkt():
    """P9: the rational map equals a direct float KKT solve of the constrained
    least-squares problem on random (non-polynomial) data."""
    rng = np.random.default_rng(7)
    # exact rows (13) and least-squares rows (4) rebuilt by quadrature of the monomials
    rows = []
    for k in range(15):
        p, q = MONOS[k]
        d, _, _ = _moments_of(lambda x, y, p=p, q=q: x ** p * y ** q)
        rows.append(d)
    A = np.array(rows).T  # 17 x 15: functional n applied to monomial k
    E, L = A[:13], A[13:]
    K = np.zeros((28, 28))
    K[:15, :15] = L.T @ L
    K[:15, 15:] = E.T
    K[15:, :15] = E
    for _ in range(5):
        d = rng.normal(size=17)
        rhs = np.concatenate([L.T @ d[13:], d[:13]])
        c = np.linalg.solve(K, rhs)[:15]
        o = O.hweno_scalar(d, linear=True)
        assert np.abs(o["c0"] - c).max() < 1e-11 * max(1.0, np.abs(c).max())


def test_weights_reduce_to_linear_weights_and_preserve_average():
    """P8: for data whose five candidates coincide (a linear field) all beta are equal,
    so omega = gamma exactly as printed (Appendix A.2); for any data the cell average
    of the nonlinear combination equals the centre average and sum(omega) = 1."""
    gold = golden_constants()
    d, _, _ = _moments_of(lambda x, y: 0.3 + 1.7 * x - 0.4 * y)
    o = O.hweno_scalar(d)
    assert np.allclose(o["omega"], [gold["gamma0"]] + [gold["gamma1_4"]] * 4, rtol=0, atol=1e-15)
    rng = np.random.default_rng(3)
    w = np.array([5 / 18, 4 / 9, 5 / 18])
    for _ in range(5):
        d = rng.normal(size=17) * rng.uniform(0.1, 10)
        o = O.hweno_scalar(d)
        assert abs(o["omega"].sum() - 1.0) < 1e-14
        vol = o["pts"][12:].reshape(3, 3)
        avg = float(w @ vol @ w)  # 3x3 Gauss is exact for the quartic combination
        assert abs(avg - d[4]) < 1e-12 * max(1, abs(d).max())


def test_nonlinear_weights_favour_the_smooth_candidate():
    """A jump across the x-direction leaves the candidates that do not straddle it
    (S1, S3 lie left and S2, S4 right of the centre) with the smallest indicators; the
    quartic's weight collapses below its linear weight."""
    d, _, _ = _moments_of(lambda x, y: np.where(x > 0.5, 1.0, 0.0))
    o = O.hweno_scalar(d)
    assert o["omega"][0] < 0.5
    assert o["beta"][1] < o["beta"][2] and o["beta"][3] < o["beta"][4]


def test_gauss_points_and_weights_match_the_paper():
    """The traces of a field linear in eta sit at the printed Gauss offsets."""
    gold = golden_constants()
    d, _, _ = _moments_of(lambda x, y: 2.0 + 3.0 * y)
    o = O.hweno_scalar(d, linear=True)
    eta = (o["pts"][:3] - 2.0) / 3.0
    assert np.allclose(eta, [-gold["gauss_node"], 0, gold["gauss_node"]], atol=1e-14)
    d, _, _ = _moments_of(lambda x, y: x ** 4)
    o = O.hweno_scalar(d, linear=True)
    w = np.array([gold["gauss_w_outer"], gold["gauss_w_centre"], gold["gauss_w_outer"]])
    # the 3-point rule integrates x^4 over the cell exactly: 1/80
    assert abs(w @ o["pts"][12:].reshape(3, 3) @ w - 1 / 80) < 1e-15


# ---------------------------------------------------------------------------
# characteristic decomposition and limiter

def test_eigenvectors_are_inverse_pairs():
    rng = np.random.default_rng(1)
    for _ in range(5):
        rho, u, v, p = rng.uniform(0.5, 2), rng.normal(), rng.normal(), rng.uniform(0.5, 2)
        ub = np.array(I.conserved(rho, u, v, p, 1.4))
        for dr in (0, 1):
            L, R = O.eigen(ub, 1.4, dr)
            assert np.abs(L @ R - np.eye(4)).max() < 1e-13
            # R diagonalises the Euler Jacobian: A r = lambda r (finite-difference Jacobian)
            c = math.sqrt(1.4 * p / rho)
            un = u if dr == 0 else v
            lam = [un - c, un, un, un + c]

            def flux(w):
                pr = 0.4 * (w[3] - 0.5 * (w[1] ** 2 + w[2] ** 2) / w[0])
                vn = w[1 + dr] / w[0]
                f = w * vn
                f[1 + dr] += pr
                f[3] += pr * vn
                return f

            J = np.zeros((4, 4))
            for k in range(4):
                e = np.zeros(4)
                e[k] = 1e-6
                J[:, k] = (flux(ub + e) - flux(ub - e)) / 2e-6
            for k in range(4):
                assert np.abs(J @ R[:, k] - lam[k] * R[:, k]).max() < 1e-7


def test_theta_root_matches_bisection():
    """P10: the quadratic-formula root equals 200-step bisection of p(t) = eps."""
    rng = np.random.default_rng(2)
    g = 1.4
    n = 0
    while n < 20:
        ub = np.array(I.conserved(rng.uniform(0.5, 2), rng.normal(), rng.normal(), rng.uniform(0.01, 1), g))
        uq = ub + rng.normal(size=4) * rng.uniform(0.5, 3)
        pq = (g - 1) * (uq[3] - 0.5 * (uq[1] ** 2 + uq[2] ** 2) / uq[0])
        if uq[0] <= 1e-3 or pq >= 1e-12:
            continue
        eps = 1e-12

        def pf(t):
            w = ub + t * (uq - ub)
            return (g - 1) * (w[3] - 0.5 * (w[1] ** 2 + w[2] ** 2) / w[0]) - eps

        lo, hi = 0.0, 1.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if pf(mid) > 0:
                lo = mid
            else:
                hi = mid
        t = O.theta_root(ub, uq, eps, g)
        assert abs(t - lo) < 1e-13
        n += 1


# ---------------------------------------------------------------------------
# whole spatial operator

def _cfg(case, **kw):
    p = case.params()
    p.update(kw)
    return O.make_cfg(**p)


def test_free_stream_is_exact():
    """P2: a constant state has zero residual (Eq. (3.2)) and is never limited."""
    for bc in (("periodic",) * 4, ("noslip", "noslip", "noslip", "symmetry")):
        case = I.Case("fs", 12, 10, bc=bc, Re=50.0)
        q = np.zeros((12, 10, 12))
        # zero velocity at walls keeps the no-slip mirror a constant state
        u, v = (0.4, -0.2) if bc[0] == "periodic" else (0.0, 0.0)
        U = I.conserved(1.3, u, v, 2.0, 1.4)
        for k in range(4):
            q[k] = U[k]
        r = O.residual(_cfg(case), q, dumps=True)
        assert np.abs(r["rhs"]).max() < 1e-13
        assert np.abs(r["vhat"]).max() < 1e-14
        assert np.all(r["theta"] == 1.0)


@pytest.mark.parametrize("kind", ["smooth", "rough"])
def test_conservation_on_periodic_grid(kind):
    """P3: on a periodic grid every face flux enters two cells with opposite signs,
    so the cell-average residual sums to zero up to round-off."""
    if kind == "smooth":
        case, q = I.random_smooth(20, 16, seed=2)
    else:
        case, q = I.random_rough(20, 16, seed=2)
    r = O.residual(_cfg(case), q)
    for v in range(4):
        scale = np.abs(r["rhs"][v]).sum()
        assert abs(r["rhs"][v].sum()) < 1e-13 * max(scale, 1.0)


def _transpose(a, ncomp):
    """x<->y transpose of moment planes: swap momenta, swap xi/eta moments."""
    perm = [0, 2, 1, 3]
    out = np.zeros((a.shape[0], a.shape[2], a.shape[1]))
    nm = a.shape[0] // 4
    for m in range(nm):
        m2 = m if (nm == 3 and m == 0) else (3 - m if nm == 3 else 1 - m)
        for v in range(4):
            out[4 * m2 + perm[v]] = a[4 * m + v].T
    return out


def _mirror_x(a):
    """x -> -x: reverse columns, flip rho*u, flip the xi-moment."""
    s = np.array([1, -1, 1, 1.0])
    out = np.zeros_like(a)
    nm = a.shape[0] // 4
    for m in range(nm):
        is_xi = (nm == 3 and m == 1) or (nm == 2 and m == 0)
        for v in range(4):
            out[4 * m + v] = (-1 if is_xi else 1) * s[v] * a[4 * m + v][:, ::-1]
    return out


@pytest.mark.parametrize("kind", ["smooth", "rough"])
def test_transpose_equivariance(kind):
    """P5: swapping x and y (with the momenta and the two moments) commutes with the
    residual, the modified moments and the wall boundaries."""
    bc = ("noslip", "symmetry", "slip", "noslip")
    if kind == "smooth":
        case, q = I.random_smooth(14, 11, seed=4, bc=bc)
    else:
        case, q = I.random_rough(14, 11, seed=4, bc=bc)
    r1 = O.residual(_cfg(case), q)
    case_t = I.Case("t", case.ny, case.nx, case.y0, case.y1, case.x0, case.x1, case.gamma, case.Pr,
                    case.Re, bc=(bc[2], bc[3], bc[0], bc[1]))
    r2 = O.residual(_cfg(case_t), _transpose(q, 12))
    a, b = _transpose(r1["rhs"], 12), r2["rhs"]
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    a, b = _transpose(r1["vhat"], 8), r2["vhat"]
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("kind", ["smooth", "rough"])
def test_mirror_equivariance(kind):
    """P5: the reflection x -> -x (rho*u and the xi-moment change sign) commutes with
    the residual; a reflective wall pair is its own image."""
    bc = ("noslip", "symmetry", "periodic", "periodic")
    if kind == "smooth":
        case, q = I.random_smooth(13, 10, seed=5, bc=bc)
    else:
        case, q = I.random_rough(13, 10, seed=5, bc=bc)
    r1 = O.residual(_cfg(case), q)
    case_m = I.Case("m", case.nx, case.ny, case.x0, case.x1, case.y0, case.y1, case.gamma, case.Pr,
                    case.Re, bc=(bc[1], bc[0], bc[2], bc[3]))
    r2 = O.residual(_cfg(case_m), _mirror_x(q))
    a, b = _mirror_x(r1["rhs"]), r2["rhs"]
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    a, b = _mirror_x(r1["vhat"]), r2["vhat"]
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_ghost_cells_follow_wall_parities():
    """Remark 4.1: at a no-slip wall both momenta are odd, rho and E even; at a
    symmetry face only the normal momentum is odd; the normal moment of a mirrored
    field changes sign relative to the tangential one."""
    case, q = I.random_smooth(8, 8, seed=1, bc=("noslip", "symmetry", "noslip", "symmetry"))
    gq = O.fill_ghosts(_cfg(case), q)
    G_ = 4
    # x-lo no-slip: ghost column G-1-k mirrors interior column k
    for k in range(4):
        gcol, icol = G_ - 1 - k, G_ + k
        for v, s in enumerate([1, -1, -1, 1]):
            assert np.allclose(gq[v, G_:-G_, gcol], s * gq[v, G_:-G_, icol])
            assert np.allclose(gq[4 + v, G_:-G_, gcol], -s * gq[4 + v, G_:-G_, icol])
            assert np.allclose(gq[8 + v, G_:-G_, gcol], s * gq[8 + v, G_:-G_, icol])
    # y-hi symmetry: ghost row ny+G+k mirrors row ny+G-1-k, rho*v odd
    ny = case.ny
    for k in range(4):
        grow, irow = ny + G_ + k, ny + G_ - 1 - k
        for v, s in enumerate([1, 1, -1, 1]):
            assert np.allclose(gq[v, grow, G_:-G_], s * gq[v, irow, G_:-G_])
            assert np.allclose(gq[4 + v, grow, G_:-G_], s * gq[4 + v, irow, G_:-G_])
            assert np.allclose(gq[8 + v, grow, G_:-G_], -s * gq[8 + v, irow, G_:-G_])


def _poly_state(n, rho_f, u_f, v_f, e_f, gamma=1.4):
    """cell moments of primitive polynomial fields on [0,1]^2 (periodic wrap only
    disturbs cells within 4 of the seam)"""
    case = I.Case("poly", n, n, gamma=gamma, Re=100.0)

    def prim(x, y):
        rho, u, v, e = rho_f(x, y), u_f(x, y), v_f(x, y), e_f(x, y)
        return rho, u, v, (gamma - 1.0) * rho * e

    return case, I.cell_moments(case, prim, nq=6)


def test_conservative_traces_exact_for_quartic_states():
    """P1 through the whole conservative path: with linear weights the characteristic
    projection is linear, so quartic conserved fields give exact traces, exact volume
    values and exact modified moments in every cell whose stencil avoids the seam."""
    n = 12
    h = 1.0 / n
    case, q = _poly_state(n, lambda x, y: 1.0 + 0 * x, lambda x, y: 0.5 + x * x - 0.3 * x * y,
                          lambda x, y: -0.2 + y * y + 0.1 * x, lambda x, y: 2.0 + x ** 4 + 0.5 * x * y ** 3)
    r = O.residual(_cfg(case, linear_weights=True, limiter=False), q, dumps=True)

    def cons(x, y):
        rho = 1.0
        u = 0.5 + x * x - 0.3 * x * y
        v = -0.2 + y * y + 0.1 * x
        e = 2.0 + x ** 4 + 0.5 * x * y ** 3
        return np.array([rho, rho * u, rho * v, rho * (e + 0.5 * (u * u + v * v))])

    for j in range(1, n - 1):
        for i in range(1, n - 1):
            xc, yc = (i + 0.5) * h, (j + 0.5) * h
            for k, (a, b) in enumerate(FACE_PTS):
                ex = cons(xc + a * h, yc + b * h)
                # E is degree 6 here? no: u^2 is degree 4, e degree 4 -> E degree 4
                assert np.abs(r["face"][4 * k:4 * k + 4, j, i] - ex).max() < 1e-11
            for k, (a, b) in enumerate(VOL_PTS):
                ex = cons(xc + a * h, yc + b * h)
                assert np.abs(r["vol"][4 * k:4 * k + 4, j, i] - ex).max() < 1e-11
            assert np.abs(r["vhat"][0:4, j, i] - q[4:8, j, i]).max() < 1e-12
            assert np.abs(r["vhat"][4:8, j, i] - q[8:12, j, i]).max() < 1e-12


def test_gradients_exact_for_polynomial_fields():
    """P7: rho = 1, u, v quadratic and e quartic (E quartic): the traces, face moments
    and 3x3 Gauss cell means are exact, so the weak-derivative moments are the exact
    moments of the derivatives (Eqs. (3.7)-(3.8)) and the linear-weight gradient
    reconstruction returns the exact derivatives at all 21 points."""
    n = 16
    h = 1.0 / n
    uf = lambda x, y: 0.5 + x * x - 0.3 * x * y + 0.2 * y * y
    vf = lambda x, y: -0.2 + y * y + 0.1 * x - 0.4 * x * x
    ef = lambda x, y: 2.0 + x ** 4 + 0.5 * x * y ** 3 - 0.7 * x * x * y
    case, q = _poly_state(n, lambda x, y: 1.0 + 0 * x, uf, vf, ef)
    r = O.residual(_cfg(case, linear_weights=True, limiter=False), q, dumps=True)

    def grads(x, y):
        return np.array([2 * x - 0.3 * y, -0.3 * x + 0.4 * y,
                         0.1 - 0.8 * x, 2 * y,
                         4 * x ** 3 + 0.5 * y ** 3 - 1.4 * x * y, 1.5 * x * y * y - 0.7 * x * x])

    for j in range(4, n - 4):
        for i in range(4, n - 4):
            xc, yc = (i + 0.5) * h, (j + 0.5) * h
            for k, (a, b) in enumerate(FACE_PTS + VOL_PTS):
                ex = grads(xc + a * h, yc + b * h)
                assert np.abs(r["grad"][6 * k:6 * k + 6, j, i] - ex).max() < 1e-9


def test_positivity_limiter_on_near_vacuum_state():
    """P4: colliding Mach-extreme streams drive traces below zero pressure; after the
    limiter every face state has rho >= eps and p >= eps (Sec. 3.1 and Sec. 5,
    eps_PP = 1e-12), theta = 1 wherever all 21 points are admissible, and only face
    values change."""
    case, q = I.colliding_streams(32, seed=3)
    cfg = _cfg(case)
    r = O.residual(cfg, q, dumps=True)
    assert r["diag"][2] > 0  # limiter engaged
    g = case.gamma
    face = r["face"].reshape(12, 4, 32, 32)
    rho = face[:, 0]
    p = (g - 1) * (face[:, 3] - 0.5 * (face[:, 1] ** 2 + face[:, 2] ** 2) / rho)
    eps = 1e-12
    assert rho.min() >= eps * (1 - 1e-9)
    assert p.min() >= eps - 1e-12 * np.abs(face[:, 3]).max()
    # cells with all points admissible are untouched
    rl = O.residual(_cfg(case, limiter=False), q, dumps=True)
    facen = rl["face"].reshape(12, 4, 32, 32)
    voln = rl["vol"].reshape(9, 4, 32, 32)
    pts = np.concatenate([facen, voln], 0)
    pp = (g - 1) * (pts[:, 3] - 0.5 * (pts[:, 1] ** 2 + pts[:, 2] ** 2) / pts[:, 0])
    ok = (pts[:, 0].min(0) >= eps) & (pp.min(0) >= eps)
    th = r["theta"]
    assert np.all(th[0][ok] == 1.0) and np.all(th[1][ok] == 1.0)
    assert np.all((th[0][~ok] < 1.0) | (th[1][~ok] < 1.0))
    assert np.array_equal(r["vol"], rl["vol"])
    assert np.array_equal(r["vhat"], rl["vhat"])


# ---------------------------------------------------------------------------
# order of accuracy of the spatial operator (Sec. 3.2 accuracy argument; Table 5.2)

def _manufactured(x, y):
    """Example 5.2's fields at t = 0 and their first derivatives."""
    tp = 2 * np.pi
    rho = 2 + 0.1 * (np.sin(tp * (2 * x - y)) + np.cos(tp * (-x + 2 * y)))
    u = 1 + 0.1 * (np.sin(tp * (-x + y)) + np.cos(tp * (x + y)))
    v = 2 + 0.1 * (np.sin(tp * (x + y)) + np.cos(tp * (x - y)))
    e = 2 + 0.1 * (np.sin(tp * (x - y)) + np.cos(tp * (x + y)))
    ux = 0.1 * tp * (-np.cos(tp * (-x + y)) - np.sin(tp * (x + y)))
    uy = 0.1 * tp * (np.cos(tp * (-x + y)) - np.sin(tp * (x + y)))
    vx = 0.1 * tp * (np.cos(tp * (x + y)) - np.sin(tp * (x - y)))
    vy = 0.1 * tp * (np.cos(tp * (x + y)) + np.sin(tp * (x - y)))
    ex = 0.1 * tp * (np.cos(tp * (x - y)) - np.sin(tp * (x + y)))
    ey = 0.1 * tp * (-np.cos(tp * (x - y)) - np.sin(tp * (x + y)))
    return rho, u, v, e, (ux, uy, vx, vy, ex, ey)


def _exact_flux(x, y, d, gamma, Pr, Re):
    rho, u, v, e, (ux, uy, vx, vy, ex, ey) = _manufactured(x, y)
    p = (gamma - 1) * rho * e
    E = rho * (e + 0.5 * (u * u + v * v))
    txx = 4 * ux / 3 - 2 * vy / 3
    txy = uy + vx
    tyy = 4 * vy / 3 - 2 * ux / 3
    if d == 0:
        return np.array([rho * u, rho * u * u + p - txx / Re, rho * u * v - txy / Re,
                         (E + p) * u - (txx * u + txy * v + gamma * ex / Pr) / Re])
    return np.array([rho * v, rho * u * v - txy / Re, rho * v * v + p - tyy / Re,
                     (E + p) * v - (txy * u + tyy * v + gamma * ey / Pr) / Re])


def _exact_rhs_avg(n, gamma, Pr, Re):
    """-(1/|K|) of the boundary integral of the exact fluxes, 8-point Gauss per face"""
    h = 1.0 / n
    gn, gw = np.polynomial.legendre.leggauss(8)
    gn, gw = 0.5 * gn, 0.5 * gw
    xc = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(xc, xc)  # [j, i]
    out = np.zeros((4, n, n))
    for a in range(8):
        fr = _exact_flux(X + 0.5 * h, Y + gn[a] * h, 0, gamma, Pr, Re)
        fl = _exact_flux(X - 0.5 * h, Y + gn[a] * h, 0, gamma, Pr, Re)
        gt = _exact_flux(X + gn[a] * h, Y + 0.5 * h, 1, gamma, Pr, Re)
        gb = _exact_flux(X + gn[a] * h, Y - 0.5 * h, 1, gamma, Pr, Re)
        out -= gw[a] * ((fr - fl) / h + (gt - gb) / h)
    return out


def test_spatial_operator_is_fifth_order():
    """P6: on Example 5.2's smooth fields the cell-average residual converges to
    the exact flux divergence at fifth order with the nonlinear weights (the scheme's
    design order, Sec. 3.2)."""
    gamma, Pr, Re = 1.4, 0.72, 100.0
    errs = []
    ns = (24, 48, 96)
    for n in ns:
        case = I.Case("mms", n, n, gamma=gamma, Pr=Pr, Re=Re)

        def prim(x, y):
            rho, u, v, e, _ = _manufactured(x, y)
            return rho, u, v, (gamma - 1) * rho * e

        q = I.cell_moments(case, prim, nq=6)
        r = O.residual(_cfg(case), q)
        err = r["rhs"][:4] - _exact_rhs_avg(n, gamma, Pr, Re)
        errs.append((np.abs(err).mean(), np.abs(err).max()))
    rates = [(math.log2(errs[k][0] / errs[k + 1][0]), math.log2(errs[k][1] / errs[k + 1][1]))
             for k in range(len(ns) - 1)]
    assert rates[-1][0] > 4.6 and rates[-1][1] > 4.5, (errs, rates)


def test_rk3_step_matches_butcher_form():
    """P13: SSP-RK3 in Shu-Osher form (Eq. (2.12)) equals the Butcher form
    k1 = F(y), k2 = F(y + dt k1), k3 = F(y + dt (k1 + k2)/4), y' = y + dt (k1 + k2 + 4 k3)/6
    on the cell averages, with each stage's first moments taken as Eq. (2.12) states
    (modified moment of the stage plus dt times the moment residual)."""
    case, q = I.random_smooth(16, 16, seed=9, Re=200.0)
    cfg = _cfg(case)
    dt = 4e-3
    r0 = O.residual(cfg, q)
    k1, vh0 = r0["rhs"], r0["vhat"]
    y1 = np.concatenate([q[:4] + dt * k1[:4], vh0 + dt * k1[4:]])
    r1 = O.residual(cfg, y1)
    k2, vh1 = r1["rhs"], r1["vhat"]
    y2 = np.concatenate([q[:4] + dt / 4 * (k1[:4] + k2[:4]), 0.75 * vh0 + 0.25 * (vh1 + dt * k2[4:])])
    r2 = O.residual(cfg, y2)
    k3 = r2["rhs"]
    avg = q[:4] + dt / 6 * (k1[:4] + k2[:4] + 4 * k3[:4])
    q1, st = O.step(cfg, q, dt_fixed=dt)
    assert st["dt"] == dt and st["rejections"] == 0
    assert np.abs(q1[:4] - avg).max() < 1e-13 * np.abs(avg).max()
    mom = vh0 / 3 + 2 / 3 * (r2["vhat"] + dt * k3[4:])
    assert np.abs(q1[4:] - mom).max() < 1e-13 * np.abs(mom).max()
    # a step that started from the evolved moments instead of the modified ones differs
    assert np.abs(vh0 - q[4:]).max() > 1e3 * 1e-13 * np.abs(mom).max()


def test_conservation_over_steps():
    """P3 over time: periodic totals of rho, rho u, rho v, E drift only by round-off."""
    case, q = I.random_rough(16, 16, seed=3)
    cfg = _cfg(case)
    tot0 = q[:4].sum(axis=(1, 2))
    q2, st = O.advance(cfg, q, 0.0, 1.0, max_steps=3)
    assert st["status"] == 0 and st["steps"] == 3
    tot1 = q2[:4].sum(axis=(1, 2))
    assert np.abs(tot1 - tot0).max() < 1e-13 * np.abs(q[:4]).sum()


def test_time_step_rule():
    """Sec. 5: dt = min(CFL h / alpha*, b Re h^2, t_end - t)."""
    case, q = I.smooth_periodic(16)
    cfg = _cfg(case)
    q1, st = O.step(cfg, q, 0.0, 10.0)
    h = 2.0 / 16
    assert st["dt"] == min(case.cfl * h / st["alpha"], case.b_visc * case.Re * h * h)
    q1, st = O.step(cfg, q, 0.0, 1e-5)
    assert st["dt"] == 1e-5
