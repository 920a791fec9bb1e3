"""Seeded synthetic workloads: cell averages and scaled first moments.

This module is shared by the CUDA path's tests and benchmark and by the oracle
tests.  It holds none of the scheme's arithmetic: it only samples primitive
point fields (rho, u, v, p) of the test problems, converts them to conserved
variables with the ideal-gas law, and integrates each cell's average and its
two scaled first moments (Sec. 3.1: u_bar, v_bar = avg(u xi), w_bar = avg(u eta))
with a 5x5 Gauss rule.

A state is a float64 array of shape (12, ny, nx): plane 4*m + v is moment m
(0 average, 1 xi-moment, 2 eta-moment) of conserved variable v
(rho, rho*u, rho*v, E).
"""
from dataclasses import dataclass, field, asdict
import math

import numpy as np

SEED_BASE = 10569


@dataclass
class Case:
    """Problem statement of one run (Sec. 3.1 model, Remark 4.1 boundaries, Sec. 5 constants)."""
    name: str
    nx: int
    ny: int
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    gamma: float = 1.4
    Pr: float = 0.72
    Re: float = 1000.0
    bc: tuple = ("periodic", "periodic", "periodic", "periodic")  # xlo, xhi, ylo, yhi
    cfl: float = 0.6
    b_visc: float = 1e-3
    eps_pp: float = 1e-12
    eps_weno: float = 1e-8
    max_halvings: int = 60
    source: int = 0          # 1: Example 5.2's manufactured source term
    inflow: tuple = None     # per side None or conserved states (A, B) of an inflow face
    band: tuple = None       # per side (centre, half-width) of the face coordinate where A applies
    t_end: float = 0.0
    extra: dict = field(default_factory=dict)

    def params(self):
        d = asdict(self)
        d.pop("name")
        d.pop("t_end")
        d.pop("extra")
        return d

    @property
    def dx(self):
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self):
        return (self.y1 - self.y0) / self.ny


_GN, _GW = np.polynomial.legendre.leggauss(5)
_GN = 0.5 * _GN          # nodes on [-1/2, 1/2]
_GW = 0.5 * _GW          # weights summing to 1


def conserved(rho, u, v, p, gamma):
    return rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)


def cell_moments(case, prim, nq=5):
    """Integrate a primitive point field prim(x, y) -> (rho, u, v, p) into
    cell averages and scaled moments with an nq x nq Gauss rule."""
    if nq == 5:
        gn, gw = _GN, _GW
    else:
        gn, gw = np.polynomial.legendre.leggauss(nq)
        gn, gw = 0.5 * gn, 0.5 * gw
    nx, ny = case.nx, case.ny
    xc = case.x0 + (np.arange(nx) + 0.5) * case.dx
    yc = case.y0 + (np.arange(ny) + 0.5) * case.dy
    q = np.zeros((12, ny, nx))
    for a in range(len(gn)):
        for b in range(len(gn)):
            X = (xc + gn[a] * case.dx)[None, :]
            Y = (yc + gn[b] * case.dy)[:, None]
            X, Y = np.broadcast_arrays(X, Y)
            U = conserved(*prim(X, Y), case.gamma)
            w = gw[a] * gw[b]
            for v in range(4):
                q[v] += w * U[v]
                q[4 + v] += w * gn[a] * U[v]
                q[8 + v] += w * gn[b] * U[v]
    return q


def _rng(k):
    return np.random.default_rng(SEED_BASE + k)


# ---------------------------------------------------------------------------
# the five benchmark workloads


def smooth_periodic(n=64, seed=1, noise=1e-3):
    """2D NS on a periodic [0,2]^2 grid: rho = 1 + 0.2 sin(pi (x+y)) plus a seeded
    uniform cell perturbation of amplitude `noise` (1e-3; 0 for the smooth field of
    convergence studies), u = 0.7, v = 0.3, p = 1, gamma 1.4, Pr 0.72, mu = 1e-3
    (Re = 1000), CFL 0.5, t_end 0.1."""
    case = Case("smooth_periodic_%d" % n, n, n, 0.0, 2.0, 0.0, 2.0, 1.4, 0.72, 1000.0,
                cfl=0.5, t_end=0.1)

    def prim(x, y):
        return 1.0 + 0.2 * np.sin(np.pi * (x + y)), 0.7 + 0 * x, 0.3 + 0 * x, 1.0 + 0 * x

    q = cell_moments(case, prim)
    d = _rng(seed).uniform(-noise, noise, size=(n, n))
    # add d to the density average keeping u, v, p of the cell fixed
    q[0] += d
    q[1] += 0.7 * d
    q[2] += 0.3 * d
    q[3] += 0.5 * d * (0.7 ** 2 + 0.3 ** 2)
    return case, q


def shock_tube(nx=1024, ny=512, Re=1000.0):
    """Viscous shock tube on [0,1] x [0,0.5]: diaphragm at x = 0.5 with
    (rho,u,v,p) = (120,0,0,120/1.4) left and (1.2,0,0,1.2/1.4) right, gamma 1.4,
    Pr 0.73, no-slip adiabatic walls at x=0, x=1, y=0, symmetry at y=0.5,
    CFL 0.3, t_end 0.2."""
    case = Case("shock_tube_%dx%d" % (nx, ny), nx, ny, 0.0, 1.0, 0.0, 0.5, 1.4, 0.73, Re,
                bc=("noslip", "noslip", "noslip", "symmetry"), cfl=0.3, t_end=0.2)
    q = np.zeros((12, ny, nx))
    xc = case.x0 + (np.arange(nx) + 0.5) * case.dx
    # the diaphragm sits on a cell face for even nx; otherwise integrate
    if nx % 2 == 0:
        left = (xc < 0.5)[None, :].repeat(ny, 0)
        rho = np.where(left, 120.0, 1.2)
        p = np.where(left, 120.0 / 1.4, 1.2 / 1.4)
        U = conserved(rho, 0 * rho, 0 * rho, p, 1.4)
        for v in range(4):
            q[v] = U[v]
    else:
        def prim(x, y):
            left = x < 0.5
            return (np.where(left, 120.0, 1.2), 0 * x, 0 * x, np.where(left, 120.0 / 1.4, 1.2 / 1.4))
        q = cell_moments(case, prim)
    return case, q


def colliding_streams(n=2048, seed=3, modes=4):
    """Low-density extreme case on a periodic [0,1]^2 grid, gamma 5/3, Re 1e4:
    rho = 1, p = 1e-4, u = -20 for x < 0.5 and +20 otherwise (the streams separate
    at x = 0.5 and collide across the periodic seam), plus a seeded smooth velocity
    noise of 1 % of 20 (a sum of `modes` low-wavenumber Fourier modes on u and v,
    peak amplitude about 0.2); t_end 0.02."""
    case = Case("colliding_streams_%d" % n, n, n, 0.0, 1.0, 0.0, 1.0, 5.0 / 3.0, 0.72, 1e4,
                cfl=0.6, t_end=0.02)
    rng = _rng(seed)
    k = rng.integers(1, 4, size=(2, modes, 2))
    a = rng.uniform(-1, 1, size=(2, modes, 2))

    def noise(x, y, f):
        s = 0 * x
        for m in range(modes):
            s = s + a[f, m, 0] * np.sin(2 * np.pi * (k[f, m, 0] * x + k[f, m, 1] * y)) \
                  + a[f, m, 1] * np.cos(2 * np.pi * (k[f, m, 1] * x + k[f, m, 0] * y))
        return 0.2 * s / modes

    def prim(x, y):
        u = np.where(x < 0.5, -20.0, 20.0) + noise(x, y, 0)
        return 1.0 + 0 * x, u, noise(x, y, 1), 1e-4 + 0 * x

    return case, cell_moments(case, prim)


def taylor_green(n, A, Re, p0, rho_pert=0.0, seed=4, gamma=1.4, name="taylor_green"):
    """Taylor-Green-type flow on [0, 2 pi]^2: u = A sin x cos y, v = -A cos x sin y,
    p = p0 + (A^2/4)(cos 2x + cos 2y), rho = 1 (+ seeded uniform cell noise)."""
    L = 2.0 * math.pi
    case = Case("%s_%d" % (name, n), n, n, 0.0, L, 0.0, L, gamma, 0.72, Re, cfl=0.6)

    def prim(x, y):
        return (1.0 + 0 * x, A * np.sin(x) * np.cos(y), -A * np.cos(x) * np.sin(y),
                p0 + 0.25 * A * A * (np.cos(2 * x) + np.cos(2 * y)))

    q = cell_moments(case, prim)
    if rho_pert > 0.0:
        d = _rng(seed).uniform(-rho_pert, rho_pert, size=(n, n))
        u = q[1] / q[0]
        v = q[2] / q[0]
        q[0] += d
        q[1] += u * d
        q[2] += v * d
        q[3] += 0.5 * d * (u * u + v * v)
    return case, q


def ensemble(ncases=64, seed=4, sizes=(128, 256, 512, 1024)):
    """64 independent periodic Taylor-Green cases: grid side drawn from sizes,
    Re log-uniform in [1e2, 1e4], amplitude A ~ U(0.1, 0.5), p0 = 1/gamma
    (unit sound speed), density cell noise of amplitude 1e-2."""
    rng = _rng(seed)
    out = []
    for k in range(ncases):
        n = int(rng.choice(sizes))
        Re = float(10 ** rng.uniform(2.0, 4.0))
        A = float(rng.uniform(0.1, 0.5))
        case, q = taylor_green(n, A, Re, 1.0 / 1.4, rho_pert=1e-2, seed=1000 + k,
                               name="ensemble%02d" % k)
        out.append((case, q))
    return out


def adjoint_taylor_green(n=512, M=0.3):
    """Taylor-Green flow for the adjoint workload: A = 1, rho = 1,
    p = 1/(gamma M^2) + (cos 2x + cos 2y)/4, Re 1600."""
    case, q = taylor_green(n, 1.0, 1600.0, 1.0 / (1.4 * M * M), name="adjoint_tg")
    return case, q


def adjoint_target(case, seed=5, modes=8, amp=0.01):
    """Seeded density target of the adjoint workload: 1 + amp times a sum of `modes`
    Fourier modes with wavenumbers |k| <= 4, sampled at the cell centres."""
    rng = _rng(seed)
    L = case.x1 - case.x0
    xc = case.x0 + (np.arange(case.nx) + 0.5) * case.dx
    yc = case.y0 + (np.arange(case.ny) + 0.5) * case.dy
    X, Y = np.meshgrid(xc, yc)
    f = np.zeros_like(X)
    for _ in range(modes):
        while True:
            kx, ky = rng.integers(-4, 5, size=2)
            if 0 < kx * kx + ky * ky <= 16:
                break
        ph = rng.uniform(0, 2 * np.pi)
        f += np.cos(2 * np.pi * (kx * X + ky * Y) / L + ph)
    return 1.0 + amp * f / modes


# ---------------------------------------------------------------------------
# generic seeded states for parity tests


def manufactured_prim(x, y, t, gamma=1.4):
    """Example 5.2's manufactured solution at time t as primitive fields (rho, u, v, p),
    with p = (gamma - 1) rho e."""
    a = 0.1 * np.exp(-t)
    tp = 2 * np.pi
    rho = 2 + a * (np.sin(tp * (2 * x - y)) + np.cos(tp * (-x + 2 * y)))
    u = 1 + a * (np.sin(tp * (-x + y)) + np.cos(tp * (x + y)))
    v = 2 + a * (np.sin(tp * (x + y)) + np.cos(tp * (x - y)))
    e = 2 + a * (np.sin(tp * (x - y)) + np.cos(tp * (x + y)))
    return rho, u, v, (gamma - 1) * rho * e


def manufactured(n, t=0.0, Re=100.0):
    """Example 5.2: [0,1]^2 periodic, gamma 1.4, Pr 0.72, Re 100, the manufactured source
    switched on, T = 0.1; the cell moments of the exact solution at time t (t = 0 the
    initial state, t = T the reference of the error table)."""
    case = Case("manufactured_%d" % n, n, n, 0.0, 1.0, 0.0, 1.0, 1.4, 0.72, Re, source=1, t_end=0.1)
    return case, cell_moments(case, lambda x, y: manufactured_prim(x, y, t, case.gamma))


def open_shock_tube(nx=1024, ny=512, Re=1000.0):
    """The viscous shock tube's box and initial state with open faces: its left state
    prescribed at x = 0 (inflow), outflow at x = 1 and y = 0.5, a symmetry plane at y = 0"""
    case, q = shock_tube(nx, ny, Re)
    left = tuple(float(v) for v in conserved(120.0, 0.0, 0.0, 120.0 / 1.4, 1.4))
    case.name = "open_shock_tube_%dx%d" % (nx, ny)
    case.bc = ("inflow", "outflow", "symmetry", "outflow")
    case.inflow = ((left, left), None, None, None)
    case.band = ((0.0, 0.0), None, None, None)
    return case, q


def sedov_2d(n, Re=1000.0):
    """Example 5.7's 2D Sedov blast: [0, 1.1]^2, rho = 1, u = v = 0, E = 0.244816/(dx dy) in
    the corner cell and 1e-12 elsewhere (gamma 1.4), reflective (symmetry) faces at x = 0
    and y = 0, outflow at x = 1.1 and y = 1.1, Re 1000, T = 1"""
    case = Case("sedov_2d_%d" % n, n, n, 0.0, 1.1, 0.0, 1.1, 1.4, 0.72, Re,
                bc=("symmetry", "outflow", "symmetry", "outflow"), t_end=1.0)
    q = np.zeros((12, n, n))
    q[0] = 1.0
    q[3] = 1e-12
    q[3, 0, 0] = 0.244816 / (case.dx * case.dy)
    return case, q


def mach2000(nx=640, ny=320, Re=1000.0):
    """Example 5.9's Mach-2000 jet: [0, 1] x [-0.25, 0.25], ambient (rho, u, v, p) =
    (0.5, 0, 0, 0.4127), gamma 5/3; inflow at x = 0 of (5, 800, 0, 0.4127) for |y| < 0.05
    and (5, 0, 0, 0.4127) elsewhere; outflow on the other sides; Re 1000, T = 0.001"""
    g = 5.0 / 3.0
    jet = conserved(5.0, 800.0, 0.0, 0.4127, g)
    still = conserved(5.0, 0.0, 0.0, 0.4127, g)
    case = Case("mach2000_%dx%d" % (nx, ny), nx, ny, 0.0, 1.0, -0.25, 0.25, g, 0.72, Re,
                bc=("inflow", "outflow", "outflow", "outflow"), t_end=0.001,
                inflow=((tuple(jet), tuple(still)), None, None, None), band=((0.0, 0.05), None, None, None))
    q = np.zeros((12, ny, nx))
    for v, val in enumerate(conserved(0.5, 0.0, 0.0, 0.4127, g)):
        q[v] = val
    return case, q


def random_smooth(nx, ny, seed=0, bc=("periodic",) * 4, gamma=1.4, Re=500.0, Pr=0.72,
                  amp=0.2, modes=3, domain=(0.0, 1.0, 0.0, 1.0)):
    """Sum of a few seeded Fourier modes on every primitive variable."""
    rng = np.random.default_rng(SEED_BASE + 100 + seed)
    case = Case("random_smooth_%dx%d_s%d" % (nx, ny, seed), nx, ny, *domain, gamma, Pr, Re, bc=tuple(bc))
    Lx, Ly = domain[1] - domain[0], domain[3] - domain[2]
    coef = rng.uniform(-1, 1, size=(4, modes, 4))
    kx = rng.integers(1, 3, size=(4, modes))
    ky = rng.integers(0, 3, size=(4, modes))
    base = np.array([1.0, 0.3, -0.2, 1.0])

    def prim(x, y):
        out = []
        for f in range(4):
            s = base[f] + 0 * x
            for m in range(modes):
                ph = 2 * np.pi * (kx[f, m] * x / Lx + ky[f, m] * y / Ly)
                s = s + amp / modes * (coef[f, m, 0] * np.sin(ph) + coef[f, m, 1] * np.cos(ph))
            out.append(s)
        return tuple(out)

    return case, cell_moments(case, prim)


def random_rough(nx, ny, seed=0, bc=("periodic",) * 4, gamma=1.4, Re=200.0, Pr=0.72,
                 jump=4.0, low=0.2):
    """Piecewise-smooth field with seeded discontinuities (a circle and a slanted
    line) and strong density/pressure contrast, to engage the nonlinear weights
    and, for small 'low', the positivity limiter."""
    rng = np.random.default_rng(SEED_BASE + 200 + seed)
    case = Case("random_rough_%dx%d_s%d" % (nx, ny, seed), nx, ny, 0.0, 1.0, 0.0, 1.0, gamma, Pr, Re,
                bc=tuple(bc))
    cx, cy, r = rng.uniform(0.3, 0.7), rng.uniform(0.3, 0.7), rng.uniform(0.15, 0.3)
    a, b = rng.uniform(-1, 1, size=2)

    def prim(x, y):
        inside = (x - cx) ** 2 + (y - cy) ** 2 < r * r
        side = (a * (x - 0.5) + b * (y - 0.5)) > 0
        rho = np.where(inside, jump, 1.0) * np.where(side, 1.0, 0.5) + low
        p = np.where(inside, jump, low * 10) + 0.05 * np.sin(2 * np.pi * x) ** 2 + low
        u = np.where(side, 0.8, -0.6) + 0.1 * np.cos(2 * np.pi * y)
        v = np.where(inside, -0.4, 0.3) + 0.1 * np.sin(2 * np.pi * x)
        return rho, u, v, p

    return case, cell_moments(case, prim)


# ---------------------------------------------------------------------------
# one-dimensional workloads (Sec. 2): states of shape (6, n), plane 3*m + v holding
# moment m (0 average, 1 scaled first moment) of v (rho, rho*u, E)

def cell_moments_1d(x0, x1, n, prim, gamma, nq=5):
    """cell averages and scaled first moments of a primitive point field
    prim(x) -> (rho, u, p) with an nq-point Gauss rule"""
    gn, gw = np.polynomial.legendre.leggauss(nq)
    gn, gw = 0.5 * gn, 0.5 * gw
    dx = (x1 - x0) / n
    xc = x0 + (np.arange(n) + 0.5) * dx
    q = np.zeros((6, n))
    for a in range(nq):
        rho, u, p = prim(xc + gn[a] * dx)
        U = (rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u)
        for v in range(3):
            q[v] += gw[a] * U[v]
            q[3 + v] += gw[a] * gn[a] * U[v]
    return q


def manufactured_prim_1d(x, t, gamma=1.4):
    """Example 5.1's manufactured solution (rho, u, p) at time t, p = (gamma - 1) rho e"""
    a = 0.2 * np.exp(-t)
    s, c = np.sin(2 * np.pi * x), np.cos(2 * np.pi * x)
    rho, u, e = 2 + a * s, 1 + a * c, 1 + a * s
    return rho, u, (gamma - 1) * rho * e


def manufactured_1d(n, t=0.0, Re=100.0):
    """Example 5.1: [0,1] periodic, gamma 1.4, Pr 0.72, Re 100, the manufactured source on,
    T = 0.1; the exact solution's cell moments at time t"""
    params = dict(n=n, x0=0.0, x1=1.0, gamma=1.4, Pr=0.72, Re=Re, bc=("periodic", "periodic"), source=1)
    return params, cell_moments_1d(0.0, 1.0, n, lambda x: manufactured_prim_1d(x, t), 1.4)


def double_rarefaction(n=200, Re=1000.0):
    """Example 5.4: [-1, 1], (rho, u, p) = (7, -1, 0.2) left of 0 and (7, 1, 0.2) right,
    gamma 1.4, Re 1000, T = 0.6, inflow (the left state) at x = -1 and outflow at x = 1;
    cell x = 0 is an interface for even n"""
    g = 1.4
    left = (7.0, -1.0 * 7.0, 0.2 / (g - 1.0) + 0.5 * 7.0)
    params = dict(n=n, x0=-1.0, x1=1.0, gamma=g, Pr=0.72, Re=Re, bc=("inflow", "outflow"),
                  inflow=(left, (0.0, 0.0, 0.0)))

    def prim(x):
        return 7.0 + 0 * x, np.where(x < 0.0, -1.0, 1.0), 0.2 + 0 * x

    return params, cell_moments_1d(-1.0, 1.0, n, prim, g)


def random_smooth_1d(n, seed=0, bc=("periodic", "periodic"), Re=300.0, amp=0.2, modes=3):
    """a few seeded Fourier modes on rho, u, p over [0, 1]"""
    rng = np.random.default_rng(SEED_BASE + 300 + seed)
    coef = rng.uniform(-1, 1, size=(3, modes, 2))
    k = rng.integers(1, 4, size=(3, modes))
    base = np.array([1.0, 0.3, 1.0])

    def prim(x):
        out = []
        for f in range(3):
            s = base[f] + 0 * x
            for m in range(modes):
                ph = 2 * np.pi * k[f, m] * x
                s = s + amp / modes * (coef[f, m, 0] * np.sin(ph) + coef[f, m, 1] * np.cos(ph))
            out.append(s)
        return tuple(out)

    params = dict(n=n, x0=0.0, x1=1.0, gamma=1.4, Pr=0.72, Re=Re, bc=tuple(bc))
    return params, cell_moments_1d(0.0, 1.0, n, prim, 1.4)
