"""SSP-RK3 steps of the 2D operator with the CUDA path's own bodies run on the host
(`host/step2d_host.cc`: the operator of `host/operator2d.h` and `rk_body`, in the order of
a handle's step), against the oracle's steps: the restart counts and step sizes of the
restart rule, the source's stage times, HWENO-DR, and runs through open faces, with the
bounds of the GPU tests.  The order of the step is restated here (the GPU tests run the
handle's own); the arithmetic and the admissibility decisions are the kernels'.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_10569_b300 import inputs as I
from parity_tools import rel_l1, rel_linf, res_tol, state_scale
from test_host_residual2d import BC, SANITIZE, open_rough, y_jet

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2608_10569_b300", "csrc")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ is needed to compile the device code for the host")
    out = str(tmp_path_factory.mktemp("step2d") / "step2d_host")
    cmd = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fno-strict-aliasing", "-I" + os.path.join(HERE, "host"),
           "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-o", out, os.path.join(HERE, "host", "step2d_host.cc")]
    if subprocess.run(cmd + SANITIZE, capture_output=True).returncode != 0:
        subprocess.check_call(cmd)
    return out


def steps(exe, tmp_path, case, q, nsteps, t=0.0, dt=0.0, mixed=False, **kw):
    """(state, status, [(dt, restarts) per step]) of the host steps"""
    p = dict(case.params(), **kw)
    nx, ny = p["nx"], p["ny"]
    inflow = p.get("inflow") or (None,) * 4
    band = p.get("band") or (None,) * 4
    st = []
    for k in range(4):
        pair = inflow[k] if inflow[k] is not None else ((0.0,) * 4, (0.0,) * 4)
        st += [float(pair[a][v]) for a in range(2) for v in range(4)]
    bd = []
    for k in range(4):
        bd += list(band[k]) if band[k] is not None else [0.0, 0.0]
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    with open(fin, "wb") as f:
        f.write(struct.pack("11i", nx, ny, *[BC[b] for b in p["bc"]], 1 if p.get("scheme") == "dr" else 0,
                            int(p.get("source", 0)), 1 if p.get("linear_grad") else 0, 0,
                            {"fused": 2, "tma": 3}.get(mixed, 1 if mixed else 0)))
        f.write(struct.pack("50d", p["x0"], p["x1"], p["y0"], p["y1"], p["gamma"], p["Pr"], p["Re"], p["eps_pp"],
                            p["eps_weno"], t, *st, *bd))
        f.write(struct.pack("i", nsteps))
        f.write(struct.pack("3d", p["cfl"], p["b_visc"], dt))
        f.write(struct.pack("i", p["max_halvings"]))
        f.write(np.ascontiguousarray(q, dtype=np.float64).tobytes())
    subprocess.check_call([exe, fin, fout])
    o = np.fromfile(fout)
    m = 12 * nx * ny
    return o[:m].reshape(12, ny, nx), int(o[m]), [(a, int(b)) for a, b in o[m + 1:].reshape(-1, 2)]


def test_restart_counts_through_the_mach2000_jet(exe, tmp_path):
    """Example 5.9 at 32 x 16 capped at 20 halvings: the oracle's restarts (2, 6, 7, 15,
    17, 18, then a step that stays inadmissible) and step sizes"""
    case, q = I.mach2000(32, 16)
    case.max_halvings = 20
    qh, status, log = steps(exe, tmp_path, case, q, 7)
    cfg = O.make_cfg(**case.params())
    qo, rows = q, []
    for _ in range(7):
        q2, st = O.step(cfg, qo)
        rows.append((st["dt"], st["rejections"]))
        if st["status"] != 0:
            break
        qo = q2
    assert status == st["status"] == -3
    assert [r for _, r in log] == [r for _, r in rows] == [2, 6, 7, 15, 17, 18, 20]
    for (a, _), (b, _) in zip(log[:6], rows[:6]):
        assert abs(a - b) <= 1e-10 * b
    assert rel_linf(qh, qo, state_scale(q)) <= res_tol(case, q)


def test_sedov_restarts_with_the_default_cap(exe, tmp_path):
    case, q = I.sedov_2d(24)
    qh, status, log = steps(exe, tmp_path, case, q, 4)
    cfg = O.make_cfg(**case.params())
    qo, t = q, 0.0
    for (dt, rej), expect in zip(log, (37, 27, 12, 7)):
        qo, st = O.step(cfg, qo, t=t)
        t += st["dt"]
        assert rej == st["rejections"] == expect and abs(dt - st["dt"]) <= 1e-6 * st["dt"]
    assert status == 0 and len(log) == 4
    assert rel_linf(qh, qo, state_scale(q)) <= res_tol(case, q)


@pytest.mark.parametrize("make", [open_rough, y_jet], ids=["open_rough", "y_jet"])
def test_runs_through_open_faces(exe, tmp_path, make):
    case, q = make()
    qh, status, log = steps(exe, tmp_path, case, q, 20)
    qo, st = O.advance(O.make_cfg(**case.params()), q, 0.0, 1e9, max_steps=20)
    assert status == 0 and len(log) == st["steps"] == 20
    assert abs(sum(a for a, _ in log) - st["t"]) <= 1e-13 * st["t"]
    assert rel_l1(qh, qo) <= 1e-9


def test_forced_step_restarts(exe, tmp_path):
    """a forced step eight times the stable size on the shock tube: three restarts to
    dt = 0.0125, as in the oracle"""
    case, q = I.shock_tube(64, 32)
    qh, status, log = steps(exe, tmp_path, case, q, 1, dt=0.1)
    qo, st = O.step(O.make_cfg(**case.params()), q, dt_fixed=0.1)
    assert status == 0 and log == [(st["dt"], st["rejections"])] == [(0.0125, 3)]
    assert rel_linf(qh, qo, state_scale(q)) <= 1e-12


@pytest.mark.parametrize("scheme", ["gr", "dr"])
def test_source_stage_times(exe, tmp_path, scheme):
    """a forced step from t = 0.02 with Example 5.2's source at t, t + dt, t + dt/2"""
    case, q = I.manufactured(24, 0.02)
    qh, status, log = steps(exe, tmp_path, case, q, 1, t=0.02, dt=1e-3, scheme=scheme)
    qo, st = O.step(O.make_cfg(**dict(case.params(), scheme=scheme)), q, t=0.02, dt_fixed=1e-3)
    assert status == 0 and log == [(1e-3, 0)]
    assert rel_linf(qh, qo, state_scale(q)) <= 1e-12


def test_dr_rule_steps(exe, tmp_path):
    case, q = I.random_rough(33, 31, seed=4, bc=("noslip", "noslip", "noslip", "symmetry"))
    qh, status, log = steps(exe, tmp_path, case, q, 2, scheme="dr")
    qo, st = O.advance(O.make_cfg(**dict(case.params(), scheme="dr")), q, 0.0, 1e9, max_steps=2)
    assert status == 0 and len(log) == 2 and abs(sum(a for a, _ in log) - st["t"]) <= 1e-13 * st["t"]
    assert rel_linf(qh, qo, state_scale(q)) <= 1e-12


def test_mixed_run_through_open_faces(exe, tmp_path):
    """the mixed path's 20 steps through the jet's inflow face: the time within 1e-6 and
    the state within 1e-5 of the oracle's FP64 run (the mixed path's wave speeds come from
    FP32 traces)"""
    case, q = y_jet()
    qh, status, log = steps(exe, tmp_path, case, q, 20, mixed=True)
    qo, st = O.advance(O.make_cfg(**case.params()), q, 0.0, 1e9, max_steps=20)
    assert status == 0 and len(log) == 20
    assert abs(sum(a for a, _ in log) - st["t"]) <= 1e-6 * st["t"]
    assert rel_l1(qh, qo) <= 1e-5


@pytest.mark.parametrize("name", ["rough_walls", "open_jet", "taylor_green"])
def test_fused_mixed_stages_equal_the_separate_kernels(exe, tmp_path, name):
    """stages 2 and 3 of a mixed step as k_flux_rk_mixed runs them (a tile's face sums in
    shared memory, then the balances and the stage update of its cells), and the
    gradients as k_grad_tma_mixed forms them, give the same steps as the separate face
    moment, weak moment, gradient, flux, balance and stage-update kernels, bit for bit:
    step sizes, restarts and states, on ragged tiles (no multiples of the tile sizes)"""
    case, q = {"rough_walls": lambda: I.random_rough(45, 23, seed=3, bc=("noslip", "noslip", "noslip", "symmetry")),
               "open_jet": y_jet,
               "taylor_green": lambda: I.taylor_green(40, 0.4, 300.0, 1 / 1.4, rho_pert=1e-2)}[name]()
    qa, sa, la = steps(exe, tmp_path, case, q, 4, mixed=True)
    qb, sb, lb = steps(exe, tmp_path, case, q, 4, mixed="fused")
    assert sa == sb == 0 and la == lb
    assert np.array_equal(qa, qb)
    # and with the gradients formed as k_grad_tma_mixed forms them (its two boxes staged,
    # zero outside the planes), in every evaluation of the step
    qc, sc, lc = steps(exe, tmp_path, case, q, 4, mixed="tma")
    assert sc == 0 and lc == la
    assert np.array_equal(qa, qc)
