"""GPU parity of HWENO-DR, of the linear-gradient ablation and of Example 5.2's source in
the batch (hweno_batch_init with such cases): the batched kernels run the single-grid
bodies, so a batch must give the handles' states (to 1e-13 of the state scale in FP64;
mixed within four times the mixed handle's distance from the FP64 handle, since the
bodies are inlined into other kernels, whose multiply-add contractions may differ) and
the oracle's steps to 1e-12.  Collected last, so that a failure here
cannot stop the other files under -x.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2608_10569_b300 import hweno, inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


def _cases():
    return [I.random_rough(37, 21, seed=2, bc=("noslip", "noslip", "noslip", "symmetry")),
            I.random_smooth(16, 16, seed=1),
            I.shock_tube(64, 32)]


@pytest.mark.parametrize("tune", [False, True])
def test_dr_batch_matches_dr_handles(tune):
    """three cases of different sizes and faces, three steps each, with and without the
    block-shape autotuning (which leaves kb_dr's block alone)"""
    cases = _cases()
    stream = torch.cuda.Stream()
    b = hweno.Batch([dict(c.params(), scheme="dr") for c, _ in cases], precision="fp64", stream=stream)
    for k, (_, q) in enumerate(cases):
        b.cases[k].set_state(q.copy())
    if tune:
        chosen = b.autotune()
        assert chosen[1] == chosen[2] == chosen[3] == -1
    for _ in range(3):
        b.step(1)
    for k, (case, q) in enumerate(cases):
        s = hweno.Solver(dict(case.params(), scheme="dr"), stream=stream)
        s.set_state(q.copy())
        for _ in range(3):
            s.step()
        ref = s.get_state().cpu().numpy()
        d = s.diag()
        s.close()
        got = b.cases[k].get_state(np.zeros_like(q))
        assert b.cases[k].diag()["steps"] == 3
        assert abs(b.cases[k].diag()["dt_last"] - d["dt_last"]) <= 1e-13 * d["dt_last"]
        scale = np.abs(q[:4]).reshape(4, -1).max(1)
        err = max(np.abs(got[j] - ref[j]).max() / max(np.abs(ref[j]).max(), scale[j % 4]) for j in range(12))
        assert err <= 1e-13, (k, err)
    b.close()


def test_dr_batch_step_matches_the_oracle():
    case, q = _cases()[0]
    p = dict(case.params(), scheme="dr")
    b = hweno.Batch([p], precision="fp64", stream=torch.cuda.Stream())
    b.cases[0].set_state(q.copy())
    b.step(1)
    qo, st = O.step(O.make_cfg(**p), q)
    got = b.cases[0].get_state(np.zeros_like(q))
    scale = np.abs(q[:4]).reshape(4, -1).max(1)
    err = max(np.abs(got[k] - qo[k]).max() / max(np.abs(qo[k]).max(), scale[k % 4]) for k in range(12))
    assert st["status"] == 0 and err <= 1e-12
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_linear_gradient_batch_matches_handles(precision):
    """Remark 3.1's ablation in a batch: three steps of three cases against the ablated
    handles; FP64 to 1e-13, mixed within four times the mixed handle's own distance from
    the FP64 handle (batches and handles compile the same FP32 expressions in different
    kernels, whose multiply-add fusions may differ)"""
    cases = _cases()
    stream = torch.cuda.Stream()
    b = hweno.Batch([dict(c.params(), linear_grad=True) for c, _ in cases], precision=precision, stream=stream)
    for k, (_, q) in enumerate(cases):
        b.cases[k].set_state(q.copy())
    for _ in range(3):
        b.step(1)

    def handle(case, q, prec):
        s = hweno.Solver(dict(case.params(), linear_grad=True), precision=prec, stream=stream)
        s.set_state(q.copy())
        for _ in range(3):
            s.step()
        out = s.get_state().cpu().numpy()
        s.close()
        return out

    def distance(a, r, q):
        scale = np.abs(q[:4]).reshape(4, -1).max(1)
        return max(np.abs(a[j] - r[j]).max() / max(np.abs(r[j]).max(), scale[j % 4]) for j in range(12))

    for k, (case, q) in enumerate(cases):
        ref = handle(case, q, precision)
        got = b.cases[k].get_state(np.zeros_like(q))
        err = distance(got, ref, q)
        bound = 1e-13 if precision == "fp64" else max(4 * distance(ref, handle(case, q, "fp64"), q), 1e-14)
        print("case %d: batch against handle %.2e, bound %.2e" % (k, err, bound))
        assert err <= bound, (k, err, bound)
    b.close()


def test_source_batch_matches_handles_and_the_oracle():
    """Example 5.2's source in a batch, with a case on a shifted domain and one without a
    source: three steps from t = 0.02 against source handles (the stage times t, t + dt,
    t + dt/2 with each case's own dt), and the first step against the oracle's"""
    t0 = 0.02
    c1, q1 = I.manufactured(24, t0)
    c2 = I.Case("manufactured_shifted_20", 20, 20, 0.3, 1.3, -0.4, 0.6, 1.4, 0.72, 100.0, source=1)
    q2 = I.cell_moments(c2, lambda x, y: I.manufactured_prim(x, y, t0, c2.gamma))
    c3, q3 = I.random_smooth(16, 16, seed=1)
    cases = [(c1, q1), (c2, q2), (c3, q3)]
    stream = torch.cuda.Stream()
    b = hweno.Batch([c.params() for c, _ in cases], precision="fp64", stream=stream)
    for k, (_, q) in enumerate(cases):
        b.cases[k].set_state(q.copy())
        b.cases[k].set_time(t0)
    b.step(1)
    first = [b.cases[k].get_state(np.zeros_like(q)) for k, (_, q) in enumerate(cases)]
    dts = [b.cases[k].diag()["dt_last"] for k in range(3)]
    for _ in range(2):
        b.step(1)
    for k, (case, q) in enumerate(cases):
        qo, st = O.step(O.make_cfg(**case.params()), q, t=t0, dt_fixed=dts[k])
        scale = np.abs(q[:4]).reshape(4, -1).max(1)
        err = max(np.abs(first[k][j] - qo[j]).max() / max(np.abs(qo[j]).max(), scale[j % 4]) for j in range(12))
        assert st["status"] == 0 and err <= 1e-12, (k, err)
        s = hweno.Solver(case.params(), stream=stream)
        s.set_state(q.copy())
        s.set_time(t0)
        for _ in range(3):
            s.step()
        ref = s.get_state().cpu().numpy()
        s.close()
        got = b.cases[k].get_state(np.zeros_like(q))
        err = max(np.abs(got[j] - ref[j]).max() / max(np.abs(ref[j]).max(), scale[j % 4]) for j in range(12))
        assert err <= 1e-13, (k, err)
    b.close()


def test_mixed_source_batch_matches_mixed_handles():
    """Example 5.2's source in a mixed batch, whose stages 2 and 3 then keep their
    residual (the flux tiles' balances, the source, then the stage update) instead of
    the fused stage kernel: three steps from t = 0.02 of two source cases and one
    without, each within four times its mixed handle's own distance from the FP64
    handle"""
    t0 = 0.02
    c1, q1 = I.manufactured(24, t0)
    c2 = I.Case("manufactured_shifted_20", 20, 20, 0.3, 1.3, -0.4, 0.6, 1.4, 0.72, 100.0, source=1)
    q2 = I.cell_moments(c2, lambda x, y: I.manufactured_prim(x, y, t0, c2.gamma))
    c3, q3 = I.random_smooth(16, 16, seed=1)
    cases = [(c1, q1), (c2, q2), (c3, q3)]
    stream = torch.cuda.Stream()
    b = hweno.Batch([c.params() for c, _ in cases], precision="mixed", stream=stream)
    for k, (_, q) in enumerate(cases):
        b.cases[k].set_state(q.copy())
        b.cases[k].set_time(t0)
    b.step(3)

    def handle(case, q, prec):
        s = hweno.Solver(case.params(), precision=prec, stream=stream)
        s.set_state(q.copy())
        s.set_time(t0)
        for _ in range(3):
            s.step()
        out = s.get_state().cpu().numpy()
        s.close()
        return out

    def distance(a, r, q):
        scale = np.abs(q[:4]).reshape(4, -1).max(1)
        return max(np.abs(a[j] - r[j]).max() / max(np.abs(r[j]).max(), scale[j % 4]) for j in range(12))

    for k, (case, q) in enumerate(cases):
        ref = handle(case, q, "mixed")
        got = b.cases[k].get_state(np.zeros_like(q))
        assert b.cases[k].diag()["steps"] == 3
        err = distance(got, ref, q)
        bound = max(4 * distance(ref, handle(case, q, "fp64"), q), 1e-14)
        print("case %d: batch against handle %.2e, bound %.2e" % (k, err, bound))
        assert err <= bound, (k, err, bound)
    b.close()
