"""GPU parity of the manufactured source (Example 5.2, hweno_config.source =
HWENO_SOURCE_MMS52): the CUDA path's residual, steps and runs with the source against
the FP64 oracle's, with the tolerances of the other parity tests (relative L-infinity
<= 1e-12 per plane after one evaluation or step, relative L1 <= 1e-9 after a run).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2608_10569_b300 import hweno, inputs as I  # noqa: E402
from test_gpu_parity import RES_TOL, flux_scale, rel_l1, rel_linf, state_scale  # noqa: E402

pytestmark = pytest.mark.gpu


def _shifted(n, t):
    """Example 5.2's fields are 1-periodic: the same problem on [0.3, 1.3] x [-0.4, 0.6],
    so that the source's coordinates come from the domain origin"""
    case = I.Case("manufactured_shifted_%d" % n, n, n, 0.3, 1.3, -0.4, 0.6, 1.4, 0.72, 100.0, source=1)
    return case, I.cell_moments(case, lambda x, y: I.manufactured_prim(x, y, t, case.gamma))


CASES = {
    "unit_24": lambda t: I.manufactured(24, t),
    "shifted_20": lambda t: _shifted(20, t),
}


def gpu_residual(params, q, t, precision="fp64"):
    s = hweno.Solver(params, precision=precision)
    s.set_state(torch.from_numpy(q).cuda())
    s.set_time(t)
    rhs, vhat = s.residual()
    out = {"rhs": rhs.cpu().numpy(), "vhat": vhat.cpu().numpy()}
    s.close()
    return out


@pytest.mark.parametrize("scheme", ["gr", "dr"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_residual_parity_with_source(name, scheme):
    t = 0.03
    case, q = CASES[name](t)
    p = dict(case.params(), scheme=scheme)
    g = gpu_residual(p, q, t)
    o = O.residual(O.make_cfg(**p, time=t), q)
    assert rel_linf(g["rhs"], o["rhs"], flux_scale(case, q)) <= RES_TOL
    assert rel_linf(g["vhat"], o["vhat"], state_scale(q)) <= RES_TOL
    # the source is not negligible here
    o0 = O.residual(O.make_cfg(**dict(p, source=0)), q)
    assert rel_linf(o["rhs"], o0["rhs"], flux_scale(case, q)) > 1e-3


def test_step_parity_with_source():
    """a forced and a rule step from t = 0.02: the stages see the source at t, t + dt,
    t + dt/2 with dt read on the device"""
    t0 = 0.02
    case, q = I.manufactured(24, t0)
    cfg = O.make_cfg(**case.params())
    s = hweno.Solver(case.params())
    s.set_state(torch.from_numpy(q).cuda())
    s.set_time(t0)
    dt, rej = s.step(1e-3)
    assert dt == 1e-3 and rej == 0
    qo, st = O.step(cfg, q, t=t0, dt_fixed=1e-3)
    assert rel_linf(s.get_state().cpu().numpy(), qo, state_scale(q)) <= 1e-12
    dt2, _ = s.step()
    qo2, st2 = O.step(cfg, qo, t=t0 + 1e-3)
    assert abs(dt2 - st2["dt"]) <= 1e-13 * st2["dt"]
    assert rel_linf(s.get_state().cpu().numpy(), qo2, state_scale(q)) <= 1e-12
    s.close()


def test_run_parity_and_accuracy_with_source():
    """32^2 to T = 0.01 under the Sec. 5 step rule: relative L1 <= 1e-9 against the
    oracle's run, and the same distance to the exact solution"""
    case, q = I.manufactured(32, 0.0)
    s = hweno.Solver(case.params())
    s.set_state(torch.from_numpy(q).cuda())
    t, n = s.advance(0.01)
    qo, st = O.advance(O.make_cfg(**case.params()), q, 0.0, 0.01)
    assert st["status"] == 0 and n == st["steps"] and abs(t - st["t"]) < 1e-15
    qg = s.get_state().cpu().numpy()
    assert rel_l1(qg, qo) <= 1e-9
    _, qex = I.manufactured(32, 0.01)
    eg, eo = np.abs(qg[0] - qex[0]).mean(), np.abs(qo[0] - qex[0]).mean()
    assert abs(eg - eo) <= 1e-6 * eo and eo < 5e-6
    s.close()


def test_mixed_precision_with_source():
    """the source is added in FP64 on the mixed path too: its residual stays within the
    mixed path's bound of the FP64 oracle"""
    t = 0.03
    case, q = I.manufactured(24, t)
    g = gpu_residual(case.params(), q, t, precision="mixed")
    o = O.residual(O.make_cfg(**case.params(), time=t), q)
    assert rel_linf(g["rhs"], o["rhs"], flux_scale(case, q)) <= 1e-5
    assert rel_linf(g["vhat"], o["vhat"], state_scale(q)) <= 1e-6


def test_the_adjoint_rejects_a_source():
    case, q = I.manufactured(16, 0.0)
    s = hweno.Solver(case.params())
    with pytest.raises(hweno.HwenoError) as e:
        s.adjoint_init()
    assert e.value.code == hweno.HWENO_ERR_ARG
    s.close()


def _table_5_2_gr():
    import os
    rows = {}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table_5_2_gr.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            n, linf, l1 = line.split()
            rows[int(n)] = (float(linf), float(l1))
    return rows


def test_example_5_2_against_table_5_2():
    """Example 5.2 with HWENO-GR to T = 0.1 at 80^2 and 120^2 under the Sec. 5 step rule:
    the density errors are of Table 5.2's size (within a factor 1.6 in both norms; the
    smoothness indicator is not printed) and fall at fifth order between the meshes"""
    tab = _table_5_2_gr()
    errs = {}
    for n in (80, 120):
        case, q = I.manufactured(n, 0.0)
        s = hweno.Solver(case.params())
        s.set_state(torch.from_numpy(q).cuda())
        t, _ = s.advance(case.t_end)
        assert t == case.t_end
        _, qex = I.manufactured(n, case.t_end)
        e = s.get_state().cpu().numpy()[0] - qex[0]
        s.close()
        errs[n] = (np.abs(e).max(), np.abs(e).mean())
        for k in range(2):
            assert tab[n][k] / 1.6 < errs[n][k] < 1.6 * tab[n][k], (n, errs[n], tab[n])
    for k in range(2):
        assert np.log(errs[80][k] / errs[120][k]) / np.log(1.5) > 4.8, errs
