"""Write the oracle's results for the step windows that the GPU window tests compare
against.  It calls only the FP64 oracle and the seeded input generators; run it from the
repository root:

    python tests/golden/make_windows.py [shock_tube] [ensemble_full] [ensemble_5]

  shock_tube_50_steps.npz   the 1024x512 viscous shock tube (no-slip walls, symmetry
                            plane, Re 1000, Pr 0.73, CFL 0.3) after 50 SSP-RK3 steps of
                            the Sec. 5 rule from its initial state: the step sizes, each
                            plane's L1 norm and sum, and every value that moved by more
                            than 1e-13 of its variable's scale (largest density, that
                            times the largest sound speed for both momenta, largest
                            energy; the moments take their variable's): the rest is the
                            initial state to that accuracy
  ensemble_full.npz         8 cases of the 64-case Taylor-Green ensemble (seeded sample of
                            the 128^2 and 256^2 cases, whose oracle runs take minutes)
                            after their 100 steps each
  ensemble_5_steps.npz      all 64 cases after 5 steps each
                            (both: per case the step sizes, each plane's L1 norm and sum,
                            and the 12 values of 64 seeded cells plus the four corners)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2608_10569_b300 import inputs as I  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
SHOCK_STEPS = 50
ENSEMBLE_STEPS = 100
ENSEMBLE_SHORT = 5
SAMPLE_CELLS = 64


def sample_cells(nx, ny, seed):
    """seeded cells of a case plus its four corners (i, j)"""
    rng = np.random.default_rng(seed)
    ci = np.concatenate([rng.integers(0, nx, SAMPLE_CELLS), [0, nx - 1, 0, nx - 1]])
    cj = np.concatenate([rng.integers(0, ny, SAMPLE_CELLS), [0, 0, ny - 1, ny - 1]])
    return ci, cj


def variable_scale(case, q):
    """per conserved variable: the largest density, that times the largest sound speed
    (both momenta), the largest total energy"""
    rho, m, n, E = q[0], q[1], q[2], q[3]
    p = (case.gamma - 1) * (E - 0.5 * (m * m + n * n) / rho)
    r = np.abs(rho).max()
    c = np.sqrt(case.gamma * p / rho).max()
    return np.array([r, r * c, r * c, np.abs(E).max()])


def full_sample():
    """the 8 cases of the full-length comparison: a seeded draw among the 128^2 and
    256^2 cases of the ensemble"""
    ens = I.ensemble(64)
    small = [k for k, (c, _) in enumerate(ens) if c.nx <= 256]
    rng = np.random.default_rng(10569 + 4)
    return sorted(int(k) for k in rng.choice(small, 8, replace=False))


def run_steps(case, q, nsteps):
    cfg = O.make_cfg(**case.params())
    dts = []
    for _ in range(nsteps):
        q, st = O.step(cfg, q)
        assert st["status"] == 0, st
        dts.append(st["dt"])
    return q, np.array(dts)


def shock_tube():
    case, q0 = I.shock_tube(1024, 512)
    t0 = time.time()
    q, dts = run_steps(case, q0.copy(), SHOCK_STEPS)
    moved = np.abs(q - q0) > 1e-13 * np.tile(variable_scale(case, q0), 3)[:, None, None]
    p, j, i = np.nonzero(moved)
    np.savez_compressed(os.path.join(HERE, "shock_tube_50_steps.npz"), dts=dts,
                        l1=np.abs(q).reshape(12, -1).sum(1), sums=q.reshape(12, -1).sum(1),
                        plane=p.astype(np.int8), j=j.astype(np.int16), i=i.astype(np.int16), value=q[p, j, i])
    print("shock tube: %d steps in %.0f s, %d moved values" % (SHOCK_STEPS, time.time() - t0, p.size), flush=True)


def ensemble(which, nsteps, name):
    ens = I.ensemble(64)
    out = {"cases": np.array(which)}
    t0 = time.time()
    for k in which:
        case, q = ens[k]
        q, dts = run_steps(case, q, nsteps)
        ci, cj = sample_cells(case.nx, case.ny, 2000 + k)
        out["dts_%02d" % k] = dts
        out["l1_%02d" % k] = np.abs(q).reshape(12, -1).sum(1)
        out["sums_%02d" % k] = q.reshape(12, -1).sum(1)
        out["cells_%02d" % k] = q[:, cj, ci]
        print("ensemble case %d (%d^2): %d steps, %.0f s so far" % (k, case.nx, nsteps, time.time() - t0),
              flush=True)
    np.savez_compressed(os.path.join(HERE, name), **out)


if __name__ == "__main__":
    what = sys.argv[1:] or ["shock_tube", "ensemble_full", "ensemble_5"]
    if "shock_tube" in what:
        shock_tube()
    if "ensemble_full" in what:
        ensemble(full_sample(), ENSEMBLE_STEPS, "ensemble_full.npz")
    if "ensemble_5" in what:
        ensemble(list(range(64)), ENSEMBLE_SHORT, "ensemble_5_steps.npz")
