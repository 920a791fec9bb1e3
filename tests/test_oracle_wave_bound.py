"""Pins of the Lax-Friedrichs coefficient (Eq. (3.3)) and of the time-step rule's alpha*
(Sec. 5) that do not restate either formula.

The PP wave-speed bound is the lemma of Zhang (J. Comput. Phys. 2017) that Eq. (3.3)
cites: for an admissible state U (rho > 0, rho e > 0) with gradients s and any
beta above the bound, both U - F(U, s)/beta and U + F(U, s)/beta are admissible,
where F is the Navier-Stokes flux (convective, viscous and heat-conduction parts) in
the face's normal direction.  Writing z = beta -+ u_n, the internal energy of the
shifted state is (z^2 rho^2 e +- z rho q - |sigma|^2/2) / beta^2 (sigma the normal
row of tau/Re - p I), so the bound is the larger root of that quadratic plus |u_n|:
admissibility holds just above it, and for states whose u_n and heat flux q have
opposite signs (or either is zero) it fails just below it.  Both directions are
checked here in exact rational arithmetic on the oracle's own bound, for random
states where the bound's positivity term dominates |u_n| + c.  Three plausible
mistakes planted in a copy of the oracle (the factor 1/2 dropped, rho for rho^2 in
the denominator, the sign of p in the normal stress) each fail one of the pins.

alpha* is the face maximum of max(|u| + c, |v| + c) with c = sqrt(gamma p / rho)
(Sec. 5): for a uniform flow every face trace is the cell average, so alpha* has the
closed form max(|u|, |v|) + c, checked for flows along either axis.
"""
import os
import shutil
import subprocess
from fractions import Fraction as Fr

import ctypes
import numpy as np
import pytest

from oracle import oracle as O

DELTA = 1e-9


def ns_flux_exact(direction, s, gr, gamma, Pr, Re):
    """the normal Navier-Stokes flux of Sec. 3.1 in exact rational arithmetic, from the
    conserved state s and the gradients gr = (u_x, u_y, v_x, v_y, e_x, e_y)"""
    rho, m, n, E = (Fr(float(a)) for a in s)
    g, Pr, Re = Fr(float(gamma)), Fr(float(Pr)), Fr(float(Re))
    ux, uy, vx, vy, ex, ey = (Fr(float(a)) for a in gr)
    u, v = m / rho, n / rho
    p = (g - 1) * (E - (m * m + n * n) / (2 * rho))
    txx = Fr(4, 3) * ux - Fr(2, 3) * vy
    txy = uy + vx
    tyy = Fr(4, 3) * vy - Fr(2, 3) * ux
    if direction == 0:
        return [m, m * u + p - txx / Re, m * v - txy / Re, (E + p) * u - (txx * u + txy * v + g * ex / Pr) / Re]
    return [n, n * u - txy / Re, n * v + p - tyy / Re, (E + p) * v - (txy * u + tyy * v + g * ey / Pr) / Re]


def admissible_shift(direction, s, gr, gamma, Pr, Re, beta, sign):
    """is U + sign F(U, s) / beta admissible (rho > 0 and rho E - |m|^2 / 2 > 0)?"""
    F = ns_flux_exact(direction, s, gr, gamma, Pr, Re)
    b = Fr(float(beta))
    w = [Fr(float(a)) + sign * f / b for a, f in zip(s, F)]
    return w[0] > 0 and w[3] * w[0] - (w[1] * w[1] + w[2] * w[2]) / 2 > 0


def sample_states(n, seed):
    """n random admissible face-point states with gradients, gas constants and Re, where
    the bound's positivity term exceeds |u_n| + c by at least 1 %"""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        gamma = float(rng.choice([1.4, 5.0 / 3.0]))
        Pr = 0.72
        Re = 10.0 ** rng.uniform(0, 3)
        rho = 10.0 ** rng.uniform(-2, 1)
        u, v = rng.uniform(-2, 2, 2)
        e = 10.0 ** rng.uniform(-3, 0)
        gr = rng.choice([-1.0, 1.0], 6) * 10.0 ** rng.uniform(-1, 3, 6)
        if rng.random() < 0.2:
            gr[rng.integers(4, 6)] = 0.0  # no heat flux in one direction
        s = np.array([rho, rho * u, rho * v, rho * (e + 0.5 * (u * u + v * v))])
        d = int(rng.integers(0, 2))
        p = (gamma - 1) * (s[3] - 0.5 * (s[1] ** 2 + s[2] ** 2) / s[0])
        c = np.sqrt(gamma * p / rho)
        cfg = O.make_cfg(4, 4, gamma=gamma, Pr=Pr, Re=Re)
        if O.wave_bound(cfg, d, s, gr) <= 1.01 * (abs((u, v)[d]) + c):
            continue
        out.append((d, s, gr, gamma, Pr, Re))
    return out


def aligned(d, s, gr):
    """u_n and the heat flux q_n of opposite signs (or one of them zero): the states for
    which the lemma's threshold is the bound itself"""
    un = s[1 + d] / s[0]
    return un * gr[4 + d] <= 0.0


def lemma_failures(states, bound):
    """(states inadmissible just above the bound, aligned states admissible just below)"""
    above, below = 0, 0
    for d, s, gr, gamma, Pr, Re in states:
        b = bound(O.make_cfg(4, 4, gamma=gamma, Pr=Pr, Re=Re), d, s, gr)
        if not all(admissible_shift(d, s, gr, gamma, Pr, Re, b * (1 + DELTA), sg) for sg in (-1, 1)):
            above += 1
        if aligned(d, s, gr) and all(admissible_shift(d, s, gr, gamma, Pr, Re, b * (1 - DELTA), sg)
                                     for sg in (-1, 1)):
            below += 1
    return above, below


STATES = None


def states():
    global STATES
    if STATES is None:
        STATES = sample_states(1200, 2017)
    return STATES


def test_wave_bound_keeps_shifted_states_admissible():
    """Zhang's lemma: U -+ F(U, s)/beta admissible for beta = (1 + 1e-9) x the bound"""
    st = states()
    assert sum(aligned(d, s, gr) for d, s, gr, *_ in st) > 300
    above, _ = lemma_failures(st, O.wave_bound)
    assert above == 0


def test_wave_bound_is_the_admissibility_threshold():
    """for states with u_n q_n <= 0, beta = (1 - 1e-9) x the bound leaves one of the two
    shifted states inadmissible: the bound is not larger than positivity needs"""
    _, below = lemma_failures(states(), O.wave_bound)
    assert below == 0


PLANTS = {
    "half dropped": ("/ (2.0 * rho * rho * e);", "/ (rho * rho * e);"),
    "rho for rho^2": ("/ (2.0 * rho * rho * e);", "/ (2.0 * rho * e);"),
    "sign of p in the normal stress": ("s1 = txx / Re - p;", "s1 = txx / Re + p;"),
}


def planted_bound(tmp_path, key):
    """the bound of a copy of the oracle with one mistake planted in its source"""
    src_dir = os.path.dirname(O._SRC)
    src = open(O._SRC).read()
    old, new = PLANTS[key]
    assert src.count(old) == 1, key
    d = tmp_path / key.replace(" ", "_").replace("^", "")
    d.mkdir()
    (d / "hweno_oracle.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(src_dir, "oracle_tables.h"), d / "oracle_tables.h")
    lib_path = d / "libplant.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", "-fopenmp",
                           "-o", str(lib_path), str(d / "hweno_oracle.c"), "-lm"])
    lib = ctypes.CDLL(str(lib_path))
    O._bind_wave_bound(lib)
    return lambda cfg, dd, s, gr: O.wave_bound(cfg, dd, s, gr, lib=lib)


@pytest.mark.parametrize("key", sorted(PLANTS))
def test_planted_bound_mistakes_fail_the_lemma(tmp_path, key):
    bound = planted_bound(tmp_path, key)
    above, below = lemma_failures(states()[:400], bound)
    assert above + below > 0, key


@pytest.mark.parametrize("vel", [(0.7, 0.3), (-0.2, 1.3), (0.0, -2.1), (3.0, 0.0)])
def test_alpha_star_of_a_uniform_flow(vel):
    """alpha* = max(|u|, |v|) + sqrt(gamma p / rho) for a uniform periodic flow"""
    rho, p, gamma = 0.8, 2.5, 1.4
    u, v = vel
    n = 6
    q = np.zeros((12, n, n))
    q[0], q[1], q[2] = rho, rho * u, rho * v
    q[3] = p / (gamma - 1) + 0.5 * rho * (u * u + v * v)
    o = O.residual(O.make_cfg(n, n, gamma=gamma), q)
    expect = max(abs(u), abs(v)) + np.sqrt(gamma * p / rho)
    assert abs(o["diag"][0] - expect) <= 4e-16 * expect
    assert np.abs(o["rhs"]).max() <= 1e-13
