"""Step windows of the workloads against the FP64 oracle, through the C ABI.

- The 1024x512 viscous shock tube, 50 SSP-RK3 steps of the Sec. 5 rule from its
  initial state: the oracle's result is stored (tests/golden/make_windows.py, which
  calls only the oracle); every cell is compared: the density's relative L1, and each
  plane's mean error against its variable's scale, to 1e-9 for the FP64 path and 1e-6
  for the mixed path (the largest error to ten times that).
- The 64-case Taylor-Green ensemble, batched: all 64 cases over 5 steps and 8 sampled
  cases over their full 100 steps, against the oracle's stored step sizes, plane L1
  norms and sums and 68 cells per case; FP64 batches to 1e-9, mixed batches to 1e-6.
- The near-vacuum colliding streams (64^2 replica, limiter engaged), 20 steps with the
  oracle run here.  The restart rule decides 20 or so admissibility checks per step on
  states with pressures clipped to eps_PP, and a rounding-level difference flips one of
  them within a few steps (the kernels' own arithmetic on the host follows the oracle's
  restarts for two steps, then takes 20 where it takes 19; on the GPU, with its
  multiply-add contractions, the first step agrees); the two runs are then different
  valid trajectories.  So the steps up to the first different restart count are
  compared cell by cell (two at most), each cell within 32 times the oracle's own spread
  there over 32 trajectories from inputs moved by one ulp (next to clipped pressures a step
  moves states by O(1) through the PP bound and can switch a face's branch; elsewhere the
  cells agree to 1e-10), and all 20 for validity: admissible states, totals conserved to
  round-off, the restarts over the 20 steps within 25 % of the oracle's and the time reached
  within a factor 10.  The mixed handle takes the FP64 route there (its internal energy is 7.5e-7
  of the total) and equals the FP64 handle bit for bit.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2608_10569_b300 import hweno, inputs as I  # noqa: E402

from parity_tools import state_scale, ulp_perturbed  # noqa: E402

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SAMPLE_CELLS = 64


def variable_scale(case, q):
    """per conserved variable: the largest density, that times the largest sound speed
    (both momenta), the largest total energy"""
    rho, m, n, E = q[0], q[1], q[2], q[3]
    p = (case.gamma - 1) * (E - 0.5 * (m * m + n * n) / rho)
    r = np.abs(rho).max()
    return np.array([r, r * np.sqrt(case.gamma * p / rho).max(), r * np.sqrt(case.gamma * p / rho).max(),
                     np.abs(E).max()])


def golden(name):
    return np.load(os.path.join(GOLDEN, name))


def sample_cells(nx, ny, seed):
    rng = np.random.default_rng(seed)
    ci = np.concatenate([rng.integers(0, nx, SAMPLE_CELLS), [0, nx - 1, 0, nx - 1]])
    cj = np.concatenate([rng.integers(0, ny, SAMPLE_CELLS), [0, 0, ny - 1, ny - 1]])
    return ci, cj


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_shock_tube_50_step_window(precision, tol):
    g = golden("shock_tube_50_steps.npz")
    case, q0 = I.shock_tube(1024, 512)
    ref = q0.copy()
    ref[g["plane"].astype(int), g["j"].astype(int), g["i"].astype(int)] = g["value"]
    s = hweno.Solver(case.params(), precision=precision)
    s.set_state(torch.from_numpy(q0).cuda())
    dts = [s.step()[0] for _ in range(len(g["dts"]))]
    q = s.get_state().cpu().numpy()
    d = s.diag()
    s.close()
    assert np.abs(np.array(dts) / g["dts"] - 1).max() <= (1e-12 if precision == "fp64" else 1e-6)
    assert d["rejected"] == 0 and d["fp64_steps"] == 0
    # every cell: the density's relative L1, and each plane's mean and largest error
    # against its variable's scale (the momentum and moment planes are near zero away
    # from the diaphragm and the walls, so their own sums are no scale)
    scale = np.tile(variable_scale(case, q0), 3)
    err = np.abs(q - ref).reshape(12, -1)
    rel_l1_rho = err[0].sum() / np.abs(ref[0]).sum()
    print("%s: density relative L1 %.2e, worst plane mean error %.2e and largest %.2e of its variable's scale"
          % (precision, rel_l1_rho, (err.mean(1) / scale).max(), (err.max(1) / scale).max()))
    assert rel_l1_rho <= tol
    assert (err.mean(1) / scale).max() <= tol
    assert (err.max(1) / scale).max() <= 10 * tol


def ensemble_run(which, nsteps, precision):
    ens = I.ensemble(64)
    cases = [ens[k] for k in which]
    b = hweno.Batch([c.params() for c, _ in cases], precision=precision)
    for view, (_, q) in zip(b.cases, cases):
        view.set_state(q)
    dts = []
    for _ in range(nsteps):
        b.step(1)
        dts.append([v.diag()["dt_last"] for v in b.cases])
    out = [v.get_state(np.zeros_like(q)) for v, (_, q) in zip(b.cases, cases)]
    b.close()
    return cases, np.array(dts).T, out


def check_ensemble(g, which, nsteps, precision, tol):
    cases, dts, states = ensemble_run(which, nsteps, precision)
    worst = 0.0
    for k, (case, q0), dt, q in zip(which, cases, dts, states):
        ref_dt = g["dts_%02d" % k]
        assert np.abs(dt / ref_dt - 1).max() <= (1e-12 if precision == "fp64" else 1e-6), k
        ci, cj = sample_cells(case.nx, case.ny, 2000 + k)
        cells = q[:, cj, ci]
        ref = g["cells_%02d" % k]
        scale = variable_scale(case, q0)
        err = max(np.abs(cells[p] - ref[p]).max() / scale[p % 4] for p in range(12))
        # plane L1 norms, against the variable's scale times the number of cells
        l1 = (np.abs(np.abs(q).reshape(12, -1).sum(1) - g["l1_%02d" % k]) / (np.tile(scale, 3) * q[0].size)).max()
        worst = max(worst, err, l1)
        assert err <= tol and l1 <= tol, (k, err, l1)
        # the average planes' sums: conservation, to FP64 round-off in both runs
        sums = q[:4].reshape(4, -1).sum(1)
        assert np.abs(sums - g["sums_%02d" % k][:4]).max() <= 1e-12 * np.abs(q0[:4]).reshape(4, -1).sum(1).max()
    return worst


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_ensemble_all_64_cases_over_5_steps(precision, tol):
    g = golden("ensemble_5_steps.npz")
    check_ensemble(g, list(g["cases"]), 5, precision, tol)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-6)])
def test_ensemble_8_cases_full_length(precision, tol):
    g = golden("ensemble_full.npz")
    check_ensemble(g, list(g["cases"]), 100, precision, tol)


def test_colliding_streams_20_step_window():
    case, q = I.colliding_streams(64)
    cfg = O.make_cfg(**case.params())
    qo, orows, ostates = q, [], []
    for _ in range(20):
        qo, st = O.step(cfg, qo)
        assert st["status"] == 0
        orows.append((st["dt"], st["rejections"]))
        ostates.append(qo)
    runs = {}
    for precision in ("fp64", "mixed"):
        s = hweno.Solver(case.params(), precision=precision)
        s.set_state(torch.from_numpy(q).cuda())
        rows, states = [], []
        for _ in range(20):
            dt, rej = s.step()
            rows.append((dt, rej))
            states.append(s.get_state().cpu().numpy())
        runs[precision] = (rows, states, s.diag())
        s.close()
    rows, states, d = runs["fp64"]
    # the mixed handle ran every step on the FP64 operator: the same result to the bit
    assert runs["mixed"][2]["fp64_steps"] == 20 and runs["mixed"][2]["max_kinetic_share"] > 1 - 1e-4
    assert runs["mixed"][0] == rows
    assert all(np.array_equal(a, b) for a, b in zip(runs["mixed"][1], states))
    # leading steps with the oracle's restart counts: cell by cell
    lead = 0
    while lead < 20 and rows[lead][1] == orows[lead][1]:
        lead += 1
    print("restarts per step: GPU %s, oracle %s; the first %d agree"
          % ([r for _, r in rows], [r for _, r in orows], lead))
    assert lead >= 1
    # next to clipped pressures a step moves states by O(1) through the PP bound (beta ~ 1/e
    # there), and a rounding-level change can switch a face's branch there (at the seam face
    # of row 19 the GPU's step differs from the oracle's by 0.38 of the variable's scale, and
    # so do two of 32 oracle runs from inputs moved by one ulp), while elsewhere the step is
    # well-conditioned.  So each cell's bound is the oracle's own spread there: its
    # trajectories from 32 inputs moved by one ulp, while their restart counts still agree,
    # per cell and per variable's scale, over the first two steps at most
    scale = np.tile(state_scale(q), 3).reshape(12, 1, 1)
    trajs = [ulp_perturbed(q, sd) for sd in range(32)]
    for k in range(min(lead, 2)):
        spread = np.zeros(q.shape[1:])
        alive = []
        for qp in trajs:
            qp, stp = O.step(cfg, qp)
            if stp["rejections"] == orows[k][1]:
                spread = np.maximum(spread, (np.abs(qp - ostates[k]) / scale).max(0))
                alive.append(qp)
        trajs = alive
        if not trajs:
            break
        err = (np.abs(states[k] - ostates[k]) / scale).max(0)
        print("step %d: GPU against the oracle %.2e, the oracle's one-ulp spread %.2e; cells within 1e-9: %d of %d"
              % (k + 1, err.max(), spread.max(), (err <= 1e-9).sum(), err.size))
        assert abs(rows[k][0] / orows[k][0] - 1) <= 1e-12
        assert (err <= 32 * spread + 1e-12).all(), np.max(err / (spread + 1e-300))
    # every step: a valid trajectory of the scheme
    area = case.dx * case.dy
    tot0 = q[:4].reshape(4, -1).sum(1) * area
    for qs in states:
        rho, m, n, E = qs[0], qs[1], qs[2], qs[3]
        assert rho.min() > 0 and (E - 0.5 * (m * m + n * n) / rho).min() > 0
        tot = qs[:4].reshape(4, -1).sum(1) * area
        assert np.abs(tot - tot0).max() <= 1e-12 * np.abs(q[:4]).reshape(4, -1).sum(1).max() * area
    # the restarts and the time reached, over the 20 steps of the two trajectories
    gr = sum(r for _, r in rows)
    orr = sum(r for _, r in orows)
    assert abs(gr / orr - 1) <= 0.25, (gr, orr)
    t_gpu, t_or = sum(dt for dt, _ in rows), sum(dt for dt, _ in orows)
    assert 0.1 < t_gpu / t_or < 10


def test_mixed_route_follows_the_kinetic_share():
    """the share a mixed handle measures at set_state is the state's own, and the ordinary
    flows stay on the FP32 operator"""
    for case, q in (I.taylor_green(48, 0.4, 300.0, 1 / 1.4, rho_pert=1e-2), I.shock_tube(64, 32),
                    I.colliding_streams(32)):
        s = hweno.Solver(case.params(), precision="mixed")
        s.set_state(torch.from_numpy(q).cuda())
        rho, m, n, E = q[0], q[1], q[2], q[3]
        share = (0.5 * (m * m + n * n) / (rho * E)).max()
        assert abs(s.diag()["max_kinetic_share"] - share) <= 1e-15
        s.step()
        s.step()
        assert s.diag()["fp64_steps"] == (2 if share > 1 - 1e-4 else 0)
        s.close()
