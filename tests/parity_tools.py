"""Tolerance helpers shared by the parity tests (CPU and GPU): the scales that relative
errors divide by, the conditioning bound of the characteristic projection, the
residual parity cases, and the oracle's own rounding floor on them."""
import numpy as np

from oracle import oracle as O
from paper_2608_10569_b300 import inputs as I

RES_TOL = 1e-12


def flux_scale(case, q):
    """per conserved variable: max over cells of (|F_v| + |G_v| + (|u| + |v| + 2c)|U_v|)/h,
    with the inviscid fluxes F, G of the cell averages and the Lax-Friedrichs
    dissipation scale: the magnitude of the face-flux terms whose differences form a
    residual plane (nonzero even for a fluid at rest).  The prescribed states of inflow
    faces enter face fluxes too, so they count among the cells."""
    g = case.gamma
    rho, m, n, E = (np.asarray(q[k], dtype=float).ravel() for k in range(4))
    inflow = getattr(case, "inflow", None) or ()
    extra = [st for pair in inflow if pair is not None for st in pair]
    if extra:
        ex = np.array(extra, dtype=float).T
        rho, m, n, E = (np.concatenate([a, ex[k]]) for k, a in enumerate((rho, m, n, E)))
    u, v = m / rho, n / rho
    p = (g - 1) * (E - 0.5 * rho * (u * u + v * v))
    c = np.sqrt(np.maximum(g * p / rho, 0.0))
    F = [m, m * u + p, m * v, (E + p) * u]
    G = [n, n * u, n * v + p, (E + p) * v]
    U = [rho, m, n, E]
    lam = np.abs(u) + np.abs(v) + 2 * c
    h = min(case.dx, case.dy)
    return np.array([(np.abs(F[k]) + np.abs(G[k]) + lam * np.abs(U[k])).max() for k in range(4)]) / h


def rel_linf(a, b, scale=None, mask=None):
    """max over planes of max|a - b| / max(max|b|, scale of the plane's variable);
    the scale guards planes that are zero up to round-off (symmetry, divergence-free
    fields), whose values are cancellation noise of much larger terms"""
    worst = 0.0
    for k in range(a.shape[0]):
        ak, bk = a[k], b[k]
        if mask is not None:
            ak, bk = ak[mask], bk[mask]
        if ak.size == 0:
            continue
        s = np.abs(bk).max()
        if scale is not None:
            s = max(s, scale[k % 4])
        d = np.abs(ak - bk).max()
        worst = max(worst, d / s if s > 0 else d)
    return worst


def state_scale(q):
    return np.abs(q[:4]).reshape(4, -1).max(1)


def char_condition(case, q, n=400):
    """largest ||L||_inf ||R||_inf of the characteristic eigenvector pairs over sampled
    cell averages and the prescribed states of inflow faces (whose ghost cells enter the
    projections next to them): rounding differences in characteristic space reach the
    traces amplified by this factor (about 1e1-1e2 for ordinary flows, 5e8 for the
    Mach-1500 colliding streams, where c ~ 0.013 and |u| = 20)"""
    ub = q[:4].reshape(4, -1).T
    idx = np.random.default_rng(0).choice(len(ub), min(n, len(ub)), replace=False)
    states = list(ub[idx])
    for pair in getattr(case, "inflow", None) or ():
        if pair is not None:
            states += [np.asarray(st, dtype=float) for st in pair]
    k = 1.0
    for u in states:
        for d in (0, 1):
            L, R = O.eigen(u, case.gamma, d)
            k = max(k, np.abs(L).sum(1).max() * np.abs(R).sum(1).max())
    return k


def res_tol(case, q):
    """1e-12, or cond * 2^-52 where the characteristic projection is ill-conditioned"""
    return max(RES_TOL, char_condition(case, q) * 2.0 ** -52)


def rel_l1(a, b):
    worst = 0.0
    for k in range(a.shape[0]):
        s = np.abs(b[k]).sum()
        d = np.abs(a[k] - b[k]).sum()
        worst = max(worst, d / s if s > 0 else d)
    return worst


# the residual parity cases: periodic, every wall type, ragged grids, the minimum grid
RESIDUAL_CASES = {
    "smooth_periodic_64": lambda: I.smooth_periodic(64),
    "rough_periodic_40x36": lambda: I.random_rough(40, 36, seed=1),
    "smooth_walls_37x29": lambda: I.random_smooth(37, 29, seed=2, bc=("noslip", "slip", "symmetry", "noslip")),
    "rough_walls_45x21": lambda: I.random_rough(45, 21, seed=3, bc=("noslip", "noslip", "noslip", "symmetry")),
    "shock_tube_64x32": lambda: I.shock_tube(64, 32),
    "taylor_green_48": lambda: I.taylor_green(48, 0.4, 300.0, 1 / 1.4, rho_pert=1e-2),
    "minimum_grid_4x4": lambda: I.random_smooth(4, 4, seed=5),
    "thin_grid_5x70": lambda: I.random_smooth(5, 70, seed=6, bc=("slip", "slip", "periodic", "periodic")),
}


def ulp_perturbed(q, seed):
    """every value moved by one unit in the last place, up or down at random"""
    rng = np.random.default_rng(seed)
    return np.nextafter(q, rng.choice([-np.inf, np.inf], size=q.shape))


def far_from(mask, r):
    """cells whose (2r+1)^2 neighbourhood (periodic) holds no True of mask"""
    out = mask.copy()
    for dj in range(-r, r + 1):
        for di in range(-r, r + 1):
            out |= np.roll(np.roll(mask, dj, 0), di, 1)
    return ~out


def oracle_floor(case, q, seeds=(0, 1, 2), mask=None):
    """the oracle's residual against itself on one-ulp perturbations of its input: the
    largest plane-relative and flux-scale-relative L-infinity differences over the seeds.
    Two correct implementations that round differently cannot be expected to agree
    more closely than this."""
    cfg = O.make_cfg(**case.params())
    r0 = O.residual(cfg, q)["rhs"]
    fs = flux_scale(case, q)
    plane = flux = 0.0
    for sd in seeds:
        r1 = O.residual(cfg, ulp_perturbed(q, sd))["rhs"]
        plane = max(plane, rel_linf(r1, r0, None, mask))
        flux = max(flux, rel_linf(r1, r0, fs, mask))
    return plane, flux
