"""Pins of the dual-number (forward-mode) build of the FP64 oracle.

That build recompiles the oracle source over dual numbers, so its tangents are only as
trustworthy as the derivative rules it adds; these checks tie them to facts outside
it: the value parts are the plain oracle's results bit for bit, the tangents agree
with Richardson-extrapolated central differences of the plain oracle (residual,
viscosity, whole step), and the residual of a uniform flow stays zero along uniform
perturbations and along the viscosity.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_10569_b300 import inputs as I


def richardson(f, h):
    """(4 D(h/2) - D(h)) / 3 with D(h) = (f(h) - f(-h)) / (2h), array-valued"""
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(h / 2) - f(-h / 2)) / h
    return (4 * d2 - d1) / 3


def _open():
    """a banded inflow face (two states, constants: no tangent), outflow and symmetry"""
    case, q = I.random_smooth(14, 12, seed=43, bc=("inflow", "outflow", "symmetry", "outflow"))
    case.inflow = ((I.conserved(1.2, 0.4, 0.1, 1.5, case.gamma), I.conserved(0.9, 0.2, 0.0, 1.1, case.gamma)),
                   None, None, None)
    case.band = ((0.5, 0.2), None, None, None)
    return case, q


CASES = {
    "walls": lambda: I.random_smooth(14, 12, seed=41, bc=("noslip", "slip", "symmetry", "noslip")),
    "periodic": lambda: I.random_smooth(12, 12, seed=42),
    "open": _open,
}


def _direction(q, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=q.shape) * np.abs(q).reshape(12, -1).max(1)[:, None, None]


@pytest.mark.parametrize("name", sorted(CASES))
def test_values_are_the_plain_oracle_bit_for_bit(name):
    case, q = CASES[name]()
    cfg = O.make_cfg(**case.params())
    v = _direction(q, 1)
    j = O.residual_jvp(cfg, q, v, dmu=1e-3)
    r = O.residual(cfg, q)
    assert np.array_equal(j["rhs"], r["rhs"])
    assert np.array_equal(j["vhat"], r["vhat"])
    q1, _, st = O.step_jvp(cfg, q, v, 1e-3, dmu=1e-3)
    q2, st2 = O.step(cfg, q, dt_fixed=1e-3)
    assert np.array_equal(q1, q2)
    assert st["status"] == 0 and st2["status"] == 0


@pytest.mark.parametrize("scheme", ["gr", "dr"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_residual_tangent_matches_differences(name, scheme):
    case, q = CASES[name]()
    cfg = O.make_cfg(**case.params(), scheme=scheme)
    v = _direction(q, 2)
    t = O.residual_jvp(cfg, q, v)["rhs_dot"]
    fd = richardson(lambda e: O.residual(cfg, q + e * v)["rhs"], 1e-6)
    assert np.abs(t - fd).max() <= 1e-8 * np.abs(t).max()
    # viscosity: mu = 1/Re
    mu0 = 1.0 / case.Re
    tm = O.residual_jvp(cfg, q, None, dmu=1.0)["rhs_dot"]

    def at(e):
        p = dict(case.params())
        p["Re"] = 1.0 / (mu0 + e)
        return O.residual(O.make_cfg(**p, scheme=scheme), q)["rhs"]

    fdm = richardson(at, 1e-2 * mu0)
    assert np.abs(tm - fdm).max() <= 1e-9 * np.abs(tm).max()


def test_step_tangent_matches_differences():
    case, q = CASES["walls"]()
    cfg = O.make_cfg(**case.params())
    v = _direction(q, 3)
    dt = 2e-3
    _, t, st = O.step_jvp(cfg, q, v, dt, dmu=0.0)
    assert st["status"] == 0 and st["rejections"] == 0
    fd = richardson(lambda e: O.step(cfg, q + e * v, dt_fixed=dt)[0], 1e-6)
    assert np.abs(t - fd).max() <= 1e-8 * np.abs(t).max()


def test_uniform_flow_has_no_tangent_along_uniform_directions():
    """a uniform state is a steady solution for every nearby uniform state and every
    viscosity, so the residual's tangent vanishes along those directions"""
    case, q = I.random_smooth(12, 12, seed=43)
    q[:] = 0.0
    q[0], q[1], q[2], q[3] = 1.2, 0.3, -0.1, 2.5
    cfg = O.make_cfg(**case.params())
    v = np.zeros_like(q)
    v[0], v[1], v[2], v[3] = 0.7, -0.2, 0.5, 1.1
    j = O.residual_jvp(cfg, q, v, dmu=1.0)
    scale = 1.0 + np.abs(q).max()
    assert np.abs(j["rhs_dot"]).max() <= 1e-12 * scale
    assert np.abs(j["vhat_dot"]).max() <= 1e-12 * scale


def test_linear_gradient_tangent_matches_differences():
    """the dual build honours Remark 3.1's ablation: its tangent with linear_grad matches
    the differences of the plain oracle's ablated residual, and differs from the
    nonlinear one"""
    case, q = _open()
    cfg = O.make_cfg(**case.params(), linear_grad=True)
    v = _direction(q, 3)
    t = O.residual_jvp(cfg, q, v)["rhs_dot"]
    fd = richardson(lambda e: O.residual(cfg, q + e * v)["rhs"], 1e-6)
    assert np.abs(t - fd).max() <= 1e-8 * np.abs(t).max()
    tn = O.residual_jvp(O.make_cfg(**case.params()), q, v)["rhs_dot"]
    assert np.abs(t - tn).max() > 1e-6 * np.abs(t).max()
