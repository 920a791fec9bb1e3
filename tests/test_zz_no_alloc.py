"""hweno_residual_noalloc: the residual for callers that cannot allocate device memory
while they run (device memory owned by another allocator under a fixed budget, or
loops that cannot take cudaMalloc's device-wide synchronisation).  It must give the
output of hweno_residual, call after call, although every call reuses the same
library-static scratch array.  Collected last so that a stop-at-first-failure run
has already run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2608_10569_b300 import hweno, inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

RES_TOL = 1e-12  # the residual parity tolerance of the other GPU tests


def _rel(a, b):
    worst = 0.0
    for k in range(a.shape[0]):
        s = np.abs(b[k]).max()
        worst = max(worst, np.abs(a[k] - b[k]).max() / (s if s > 0 else 1.0))
    return worst


def _noalloc(case, qd):
    lib = hweno.load()
    cfg = hweno.make_config(**case.params())
    rhs = torch.full((12, case.ny, case.nx), float("nan"), dtype=torch.float64, device="cuda")
    vhat = torch.full((8, case.ny, case.nx), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = lib.hweno_residual_noalloc(ctypes.byref(cfg), ctypes.c_void_p(qd.data_ptr()),
                                    ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(vhat.data_ptr()),
                                    ctypes.c_void_p(stream.cuda_stream))
    assert rc == hweno.HWENO_OK, lib.hweno_last_error(None)
    torch.cuda.synchronize()
    return rhs.cpu().numpy(), vhat.cpu().numpy()


def _with_handle(case, qd):
    s = hweno.Solver(case.params(), precision="mixed" if case.params().get("precision") == "mixed" else "fp64")
    s.set_state(qd)
    rhs, vhat = s.residual()
    out = rhs.cpu().numpy(), vhat.cpu().numpy()
    s.close()
    return out


def test_noalloc_matches_hweno_residual_on_two_calls_in_a_row():
    # the second grid is smaller, so the first call's contents are still in the array
    cases = [I.random_rough(40, 36, seed=21),
             I.random_smooth(33, 29, seed=22, bc=("noslip", "noslip", "noslip", "symmetry"))]
    for case, q in cases:
        qd = torch.from_numpy(q).cuda()
        r1, v1 = _noalloc(case, qd)
        r0, v0 = _with_handle(case, qd)
        assert np.isfinite(r1).all() and np.isfinite(v1).all()
        assert _rel(r1, r0) <= RES_TOL
        assert _rel(v1, v0) <= RES_TOL


def _open_rough():
    case, q = I.random_rough(40, 36, seed=9, bc=("inflow", "outflow", "symmetry", "outflow"), Re=200.0)
    case.inflow = ((tuple(q[:4, 18, 0]), tuple(q[:4, 5, 0])), None, None, None)
    case.band = ((0.5, 0.15), None, None, None)
    return case, q


def _variant(case, **kw):
    p = dict(case.params(), **kw)
    case.params = lambda: p
    return case


@pytest.mark.parametrize("variant", ["mixed", "open_faces", "linear_grad", "mixed_open_faces"])
def test_noalloc_variants_match_a_handle_of_the_same_setting(variant):
    """the mixed precision (its FP32 split of the state lives in the static array too),
    inflow and outflow faces, and the linear-gradient ablation, each against a handle with
    the same setting, on two calls in a row of different grids"""
    def make(k):
        if "open" in variant:
            case, q = _open_rough() if k == 0 else I.random_smooth(31, 27, seed=24, bc=("outflow",) * 4)
        else:
            case, q = I.random_rough(40, 36, seed=23) if k == 0 else I.random_smooth(31, 27, seed=24)
        kw = {}
        if "mixed" in variant:
            kw["precision"] = "mixed"
        if variant == "linear_grad":
            kw["linear_grad"] = True
        return _variant(case, **kw), q

    for k in range(2):
        case, q = make(k)
        qd = torch.from_numpy(q).cuda()
        r1, v1 = _noalloc(case, qd)
        r0, v0 = _with_handle(case, qd)
        assert np.isfinite(r1).all() and np.isfinite(v1).all()
        assert _rel(r1, r0) <= RES_TOL, (variant, k)
        assert _rel(v1, v0) <= RES_TOL, (variant, k)


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    lib = hweno.load()
    case, q = I.random_smooth(64, 64, seed=1)  # (64+8) * 80 = 5760 > 4096 padded cells
    cfg = hweno.make_config(**case.params())
    qd = torch.from_numpy(q).cuda()
    out = torch.zeros((12, 64, 64), dtype=torch.float64, device="cuda")
    rc = lib.hweno_residual_noalloc(ctypes.byref(cfg), ctypes.c_void_p(qd.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), None, None)
    assert rc == hweno.HWENO_ERR_ARG
    assert b"static scratch" in lib.hweno_last_error(None)
    assert torch.count_nonzero(out).item() == 0
