"""GPU parity of HWENO-DR (hweno_config.scheme = HWENO_SCHEME_DR): the CUDA path
(k_cons_dr storing the characteristic combinations, k_dr differentiating them) against
the FP64 oracle's DR gradients on the same seeded inputs, with the tolerances of the
HWENO-GR parity tests: relative L-infinity <= 1e-12 per plane after one evaluation,
relative L1 <= 1e-9 after a full run.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2608_10569_b300 import hweno, inputs as I  # noqa: E402
from test_gpu_parity import (RES_TOL, _sample_cells, flux_scale, rel_l1, rel_linf, res_tol,  # noqa: E402
                             state_scale)

pytestmark = pytest.mark.gpu


def dr(params, **kw):
    p = dict(params)
    p["scheme"] = "dr"
    p.update(kw)
    return p


def gpu_residual(params, q, dumps=()):
    s = hweno.Solver(params)
    s.set_state(torch.from_numpy(q).cuda())
    rhs, vhat = s.residual()
    out = {"rhs": rhs.cpu().numpy(), "vhat": vhat.cpu().numpy(), "diag": s.diag()}
    for w in dumps:
        out[w] = s.debug_fields(w).cpu().numpy()
    s.close()
    return out


CASES = {
    "smooth_periodic_64": lambda: I.smooth_periodic(64),
    "rough_periodic_40x36": lambda: I.random_rough(40, 36, seed=1),
    "smooth_walls_37x29": lambda: I.random_smooth(37, 29, seed=2, bc=("noslip", "slip", "symmetry", "noslip")),
    "rough_walls_45x21": lambda: I.random_rough(45, 21, seed=3, bc=("noslip", "noslip", "noslip", "symmetry")),
    "shock_tube_64x32": lambda: I.shock_tube(64, 32),
    "taylor_green_48": lambda: I.taylor_green(48, 0.4, 300.0, 1 / 1.4, rho_pert=1e-2),
    "minimum_grid_4x4": lambda: I.random_smooth(4, 4, seed=5),
    "thin_grid_5x70": lambda: I.random_smooth(5, 70, seed=6, bc=("slip", "slip", "periodic", "periodic")),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_residual_parity(name):
    case, q = CASES[name]()
    g = gpu_residual(dr(case.params()), q)
    o = O.residual(O.make_cfg(**dr(case.params())), q)
    assert res_tol(case, q) == RES_TOL
    assert rel_linf(g["rhs"], o["rhs"], flux_scale(case, q)) <= RES_TOL
    assert rel_linf(g["vhat"], o["vhat"], state_scale(q)) <= RES_TOL
    assert abs(g["diag"]["alpha_star"] - o["diag"][0]) <= 1e-13 * o["diag"][0]
    assert abs(g["diag"]["beta_max"] - o["diag"][1]) <= 1e-12 * o["diag"][1]


def test_gradient_parity():
    """the DR gradients at the 21 points, with the traces and volume values they use"""
    case, q = I.random_rough(40, 36, seed=7, bc=("noslip", "symmetry", "periodic", "periodic"))
    g = gpu_residual(dr(case.params()), q, dumps=(0, 1, 3))
    o = O.residual(O.make_cfg(**dr(case.params())), q, dumps=True)
    assert rel_linf(g[0], o["face"], state_scale(q)) <= RES_TOL
    assert rel_linf(g[1], o["vol"], state_scale(q)) <= RES_TOL
    assert rel_linf(g[3], o["grad"]) <= RES_TOL
    # DR's gradients are not GR's (the comparison is not vacuous)
    o_gr = O.residual(O.make_cfg(**case.params()), q, dumps=True)
    assert rel_linf(g[3], o_gr["grad"]) > 1e-6


@pytest.mark.parametrize("name", ["rough_walls_45x21", "shock_tube_64x32"])
def test_euler_limit_dr_equals_gr(name):
    """with 1/Re = 0 the viscous fluxes vanish and the two schemes share everything
    else: the GPU's DR and GR residuals agree to rounding (the trace kernels are two
    compilations of one body), and both match the oracle"""
    case, q = CASES[name]()
    p = dict(case.params(), Re=math.inf)
    g_gr = gpu_residual(p, q)
    g_dr = gpu_residual(dr(p), q)
    scale = flux_scale(case, q)
    assert rel_linf(g_dr["rhs"], g_gr["rhs"], scale) <= 1e-14
    assert rel_linf(g_dr["vhat"], g_gr["vhat"], state_scale(q)) <= 1e-14
    o = O.residual(O.make_cfg(**dr(p)), q)
    assert rel_linf(g_dr["rhs"], o["rhs"], scale) <= RES_TOL


def test_full_size_sampled_parity_shock_tube():
    """the benchmark's 1024 x 512 shock tube in its launch configuration, sampled cells
    (the diaphragm densely) checked one by one against the oracle"""
    case, q = I.shock_tube(1024, 512)
    g = gpu_residual(dr(case.params()), q, dumps=(4,))
    ci, cj = _sample_cells(case, 300, 98)
    ci = np.concatenate([ci, np.full(64, case.nx // 2 - 1), np.full(64, case.nx // 2)])
    cj = np.concatenate([cj, np.arange(64) * (case.ny // 64), np.arange(64) * (case.ny // 64)])
    rhs, vh = O.residual_cells(O.make_cfg(**dr(case.params())), q, ci, cj)
    limited = (g[4][0] < 1) | (g[4][1] < 1)
    keep = np.array([not limited[max(0, j - 4):j + 5, max(0, i - 4):i + 5].any() for i, j in zip(ci, cj)])
    assert keep.sum() > 0.5 * len(ci)
    tol = res_tol(case, q)
    assert rel_linf(g["rhs"][:, cj, ci][:, keep], rhs.T[:, keep], flux_scale(case, q)) <= tol
    assert rel_linf(g["vhat"][:, cj, ci], vh.T, state_scale(q)) <= tol


def test_step_parity():
    case, q = I.random_rough(33, 31, seed=4, bc=("noslip", "noslip", "noslip", "symmetry"))
    cfg = O.make_cfg(**dr(case.params()))
    s = hweno.Solver(dr(case.params()))
    s.set_state(torch.from_numpy(q).cuda())
    dt, rej = s.step(2e-3)
    assert dt == 2e-3 and rej == 0
    qo, _ = O.step(cfg, q, dt_fixed=2e-3)
    assert rel_linf(s.get_state().cpu().numpy(), qo, state_scale(q)) <= 1e-12
    dt2, _ = s.step()
    qo2, st2 = O.step(cfg, qo)
    assert abs(dt2 - st2["dt"]) <= 1e-13 * st2["dt"]
    assert rel_linf(s.get_state().cpu().numpy(), qo2, state_scale(q)) <= 1e-12
    s.close()


def test_full_run_smooth_periodic():
    """64^2 periodic flow to t = 0.1 under the Sec. 5 time-step rule with DR gradients:
    relative L1 <= 1e-9 against the oracle's DR run, totals conserved"""
    case, q = I.smooth_periodic(64)
    s = hweno.Solver(dr(case.params()))
    s.set_state(torch.from_numpy(q).cuda())
    t, n = s.advance(case.t_end)
    qo, st = O.advance(O.make_cfg(**dr(case.params())), q, 0.0, case.t_end)
    assert st["status"] == 0 and n == st["steps"] and abs(t - st["t"]) < 1e-15
    assert rel_l1(s.get_state().cpu().numpy(), qo) <= 1e-9
    d = s.diag()
    tot0 = q[:4].sum(axis=(1, 2)) * case.dx * case.dy
    assert np.abs(np.array(d["totals"]) - tot0).max() <= 1e-13 * np.abs(tot0).max()
    s.close()


def test_gr_only_entry_points_reject_dr():
    """the adjoint is written for HWENO-GR, and a batch runs one scheme: a DR handle's
    adjoint and a batch mixing GR and DR cases are refused with HWENO_ERR_ARG, not run
    with the wrong gradients"""
    case, q = I.random_smooth(16, 16, seed=1)
    s = hweno.Solver(dr(case.params()))
    with pytest.raises(hweno.HwenoError) as e:
        s.adjoint_init()
    assert e.value.code == hweno.HWENO_ERR_ARG
    s.close()
    with pytest.raises(hweno.HwenoError) as e:
        hweno.Batch([case.params(), dr(case.params())], precision="fp64")
    assert e.value.code == hweno.HWENO_ERR_ARG
