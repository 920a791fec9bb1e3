"""Batched ensembles (hweno_batch_*): every case of a batch must follow the steps its own
single-grid solver takes (same per-cell bodies, same per-case time step), also after the
autotuner changed the tile shapes, and with per-case restarts: in FP64 bit for bit.  In
the mixed path a batch runs the handles' FP32 expressions in its own kernels (the
TMA-staged gradient pass over its work list, the flux tile kernels); a multiply and an
add written without a rounding mode may be fused into one multiply-add by the code
generator, differently in different kernels, so a mixed batch and a mixed handle agree
to FP32 rounding: their distance is bounded by the mixed
handle's own distance from the FP64 handle on the same case."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2608_10569_b300 import hweno, inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


def _cases():
    return [I.random_smooth(16, 16, seed=1),
            I.random_rough(37, 21, seed=2, bc=("noslip", "noslip", "noslip", "symmetry")),
            I.taylor_green(32, 0.3, 500.0, 1 / 1.4, rho_pert=1e-2, seed=7),
            I.random_smooth(24, 40, seed=3, bc=("slip", "symmetry", "periodic", "periodic")),
            I.shock_tube(48, 24)]


def _single(case, q, precision, nsteps):
    s = hweno.Solver(case.params(), precision=precision)
    s.set_state(torch.from_numpy(q).cuda())
    dts = [s.step()[0] for _ in range(nsteps)]
    out = s.get_state().cpu().numpy(), dts, s.diag()
    s.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("tune", [False, True])
def test_batch_matches_single_solvers(precision, tune):
    cases = _cases()
    stream = torch.cuda.Stream()
    b = hweno.Batch([c.params() for c, _ in cases], precision=precision, stream=stream)
    with torch.cuda.stream(stream):
        for view, (case, q) in zip(b.cases, cases):
            view.set_state(torch.from_numpy(q).cuda())
    stream.synchronize()
    if tune:
        chosen = b.autotune()
        # a mixed batch's fluxes and (TMA-staged) gradient kinds run in fixed tiles: not tuned
        fixed = (1, 2, 3, 4) if precision == "mixed" else ()
        assert len(chosen) == 6 and all(0 <= c < 4 for k, c in enumerate(chosen) if k not in fixed)
        assert all(chosen[k] == -1 for k in fixed)
    n0 = b.launch_count()
    assert b.step(3) == 0
    assert b.launch_count() > n0
    for view, (case, q) in zip(b.cases, cases):
        ref, dts, d1 = _single(case, q, precision, 3)
        with torch.cuda.stream(stream):
            got = view.get_state().cpu().numpy()
        stream.synchronize()
        d = view.diag()
        if precision == "fp64":
            assert d["steps"] == 3 and d["dt_last"] == dts[-1]
            assert abs(d["t"] - sum(dts)) <= 1e-15 * sum(dts)
            assert np.array_equal(got, ref)
        else:
            assert d["steps"] == 3 and abs(d["dt_last"] / dts[-1] - 1) <= 1e-6
            assert abs(d["t"] / sum(dts) - 1) <= 1e-6
            ref64 = _single(case, q, "fp64", 3)[0]
            bound = mixed_distance(ref, ref64, q)
            err = mixed_distance(got, ref, q)
            print("%s: batch against handle %.2e, mixed handle against FP64 %.2e" % (case.name, err, bound))
            assert err <= max(4 * bound, 1e-14)
    b.close()


def mixed_distance(a, b, q):
    """max over planes of max |a - b| against the plane's variable's scale"""
    scale = np.abs(q[:4]).reshape(4, -1).max(1)
    return max(np.abs(a[k] - b[k]).max() / max(np.abs(b[k]).max(), scale[k % 4]) for k in range(12))


def test_batch_fp64_matches_the_oracle():
    case, q = I.random_rough(37, 21, seed=2, bc=("noslip", "noslip", "noslip", "symmetry"))
    b = hweno.Batch([case.params(), I.random_smooth(16, 16, seed=1)[0].params()], precision="fp64",
                    stream=torch.cuda.Stream())
    b.cases[0].set_state(q.copy())
    b.cases[1].set_state(I.random_smooth(16, 16, seed=1)[1])
    b.step(1)
    qo, st = O.step(O.make_cfg(**case.params()), q)
    got = b.cases[0].get_state(np.zeros_like(q))
    scale = np.abs(q[:4]).reshape(4, -1).max(1)
    err = max(np.abs(got[k] - qo[k]).max() / max(np.abs(qo[k]).max(), scale[k % 4]) for k in range(12))
    assert err <= 1e-12
    b.close()


def test_batch_restarts_only_the_rejected_case():
    """A shock tube whose CFL number is far above the stable one is rejected and
    repeated with half its step (Sec. 5) while the other case advances once; both end
    where their single-grid solvers end."""
    fast, qf = I.shock_tube(48, 24)
    fast.cfl = 8.0
    fast.b_visc = 10.0
    calm, qc = I.random_smooth(20, 20, seed=4)
    b = hweno.Batch([fast.params(), calm.params()], precision="fp64", stream=torch.cuda.Stream())
    b.cases[0].set_state(qf.copy())
    b.cases[1].set_state(qc.copy())
    rej = b.step(1)
    assert rej > 0
    for view, (case, q) in zip(b.cases, [(fast, qf), (calm, qc)]):
        s = hweno.Solver(case.params())
        s.set_state(q.copy())
        s.step()
        ref = s.get_state(np.zeros_like(q))
        s.close()
        assert np.array_equal(view.get_state(np.zeros_like(q)), ref)
    assert b.cases[0].diag()["rejected"] == rej and b.cases[1].diag()["rejected"] == 0
    b.close()


def test_mixed_batch_restarts_only_the_rejected_case():
    """The same pair in the mixed path over three steps: the rejected case's stage 1
    splits its state again on each retry (the attempt's stage updates overwrote the
    split), the accepted cases reuse the split their last stage-3 update wrote.  Each case
    ends with its mixed single-grid solver's restarts, within FP32 rounding of its state
    (four times the mixed solver's own distance from the FP64 solver)."""
    fast, qf = I.shock_tube(48, 24)
    fast.cfl = 8.0
    fast.b_visc = 10.0
    calm, qc = I.random_smooth(20, 20, seed=4)
    b = hweno.Batch([fast.params(), calm.params()], precision="mixed", stream=torch.cuda.Stream())
    b.cases[0].set_state(qf.copy())
    b.cases[1].set_state(qc.copy())
    rej = b.step(3)
    assert rej > 0
    for view, (case, q) in zip(b.cases, [(fast, qf), (calm, qc)]):
        out = {}
        for prec in ("mixed", "fp64"):
            s = hweno.Solver(case.params(), precision=prec)
            s.set_state(q.copy())
            for _ in range(3):
                s.step()
            out[prec] = (s.get_state(np.zeros_like(q)), s.diag())
            s.close()
        got = view.get_state(np.zeros_like(q))
        assert view.diag()["steps"] == 3 and view.diag()["rejected"] == out["mixed"][1]["rejected"]
        err = mixed_distance(got, out["mixed"][0], q)
        bound = mixed_distance(out["mixed"][0], out["fp64"][0], q)
        print("%s: batch against handle %.2e, mixed handle against FP64 %.2e" % (case.name, err, bound))
        assert err <= max(4 * bound, 1e-14)
        # the case's own residual reuses the split the batch's last update wrote: the same
        # kernels on the same split as a fresh handle, which splits the state itself
        rhs_view = view.residual()[0]
        torch.cuda.synchronize()  # the view works on the batch's stream
        rhs_view = rhs_view.cpu().numpy()
        s = hweno.Solver(case.params(), precision="mixed")
        s.set_state(got.copy())
        rhs_fresh = s.residual()[0]
        torch.cuda.synchronize()
        assert np.array_equal(rhs_view, rhs_fresh.cpu().numpy())
        s.close()
    assert b.cases[0].diag()["rejected"] == rej and b.cases[1].diag()["rejected"] == 0
    b.close()


def test_mixed_batch_beyond_the_tensor_map_limit():
    """A mixed batch of more cases than its kernel parameter holds tensor maps for (64)
    runs its face moments, weak moments and gradients in the separate work-list kernels,
    whose block shapes the autotuner then picks: 65 small cases of mixed sizes and
    faces, two steps after tuning, each within four times its mixed handle's own
    distance from the FP64 handle of that handle's state"""
    bcs = [("periodic",) * 4, ("noslip", "noslip", "noslip", "symmetry"), ("slip", "symmetry", "periodic", "periodic")]
    cases = [I.random_smooth(8 + k % 7, 6 + (3 * k) % 9, seed=200 + k, bc=bcs[k % 3]) for k in range(65)]
    stream = torch.cuda.Stream()
    b = hweno.Batch([c.params() for c, _ in cases], precision="mixed", stream=stream)
    for view, (_, q) in zip(b.cases, cases):
        view.set_state(q.copy())
    chosen = b.autotune()
    assert chosen[4] == -1 and all(0 <= chosen[k] < 4 for k in (0, 1, 2, 3, 5))
    assert b.step(2) == 0
    worst = 0.0
    for view, (case, q) in zip(b.cases, cases):
        out = {}
        for prec in ("mixed", "fp64"):
            s = hweno.Solver(case.params(), precision=prec, stream=stream)
            s.set_state(q.copy())
            for _ in range(2):
                s.step()
            out[prec] = s.get_state(np.zeros_like(q))
            s.close()
        got = view.get_state(np.zeros_like(q))
        assert view.diag()["steps"] == 2
        err = mixed_distance(got, out["mixed"], q)
        bound = mixed_distance(out["mixed"], out["fp64"], q)
        worst = max(worst, err / max(bound, 1e-300))
        assert err <= max(4 * bound, 1e-14), (case.name, err, bound)
    print("worst batch-against-handle distance over the handle's distance from FP64: %.2f" % worst)
    b.close()


def test_ensemble_case_against_the_oracle_at_full_length():
    """The 64-case ensemble's first 128^2 case, stepped by the batch for its 100 steps
    in FP64 and in mixed precision, against the FP64 oracle run at the batch's step
    sizes: FP64 to 1e-9 relative L1 (the full-run bar), mixed to 1e-6."""
    case, q = next((c, q) for c, q in I.ensemble(64) if c.nx == 128)
    out, dts = {}, None
    for prec in ("fp64", "mixed"):
        b = hweno.Batch([case.params()], precision=prec, stream=torch.cuda.Stream())
        b.cases[0].set_state(q)
        steps = []
        for _ in range(100):
            b.step(1)
            steps.append(b.cases[0].diag()["dt_last"])
        out[prec] = b.cases[0].get_state(np.zeros_like(q))
        b.close()
        if prec == "fp64":
            dts = steps
    cfg = O.make_cfg(**case.params())
    ref = q
    for dt in dts:
        ref, st = O.step(cfg, ref, dt_fixed=dt)
        assert st["status"] == 0 and st["rejections"] == 0
    for prec, bound in (("fp64", 1e-9), ("mixed", 1e-6)):
        for k in range(12):
            err = np.abs(out[prec][k] - ref[k]).sum() / max(np.abs(ref[k]).sum(), np.abs(ref[:4]).sum(axis=(1, 2)).max())
            assert err <= bound, (prec, k, err)
