"""The 2D spatial operator of the CUDA path run on the host, against the FP64 oracle.

`host/residual2d_host.cc` compiles the kernels' own code (`hweno_state.cuh`,
`hweno_ops.cuh`, `hweno_mixed.cuh`, `hweno_source.cuh`) as plain C++ with `host/shim.h`
and calls every kernel body of the FP64 operator, or of the mixed FP32/FP64 one, over
the index range of its launch, in the operator's order, with one host thread standing
for each thread block.  Every scratch plane starts as NaN, so an
operator that read a value no earlier kernel wrote would not match; every plane set is
its own allocation, checked by AddressSanitizer and UBSan where the compiler has them.
The tolerances are those of the GPU parity tests: relative L-infinity 1e-12 of the flux
scale per residual plane (the conditioning bound where the characteristic projection
is ill-conditioned), 1e-5 on the mixed path.  What this cannot check, the GPU's own arithmetic and the
interleaving of threads, the GPU parity tests cover.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_10569_b300 import inputs as I
from parity_tools import flux_scale, rel_linf, res_tol, state_scale

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2608_10569_b300", "csrc")
SANITIZE = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-g"]
BC = {"periodic": 0, "noslip": 1, "symmetry": 2, "slip": 3, "inflow": 4, "outflow": 5}


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ is needed to compile the device code for the host")
    out = str(tmp_path_factory.mktemp("residual2d") / "residual2d_host")
    # the mixed path's float planes live in the double scratch planes
    cmd = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fno-strict-aliasing", "-I" + os.path.join(HERE, "host"),
           "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-o", out, os.path.join(HERE, "host", "residual2d_host.cc")]
    if subprocess.run(cmd + SANITIZE, capture_output=True).returncode != 0:
        subprocess.check_call(cmd)
    return out


def write_header(f, p, t=0.0, mixed=False):
    """the configuration record of host/operator2d.h (NaN-filled scratch)"""
    inflow = p.get("inflow") or (None,) * 4
    band = p.get("band") or (None,) * 4
    st = []
    for k in range(4):
        pair = inflow[k] if inflow[k] is not None else ((0.0,) * 4, (0.0,) * 4)
        st += [float(pair[a][v]) for a in range(2) for v in range(4)]
    bd = []
    for k in range(4):
        bd += list(band[k]) if band[k] is not None else [0.0, 0.0]
    f.write(struct.pack("11i", p["nx"], p["ny"], *[BC[b] for b in p["bc"]], 1 if p.get("scheme") == "dr" else 0,
                        int(p.get("source", 0)), 1 if p.get("linear_grad") else 0, 1, int(mixed)))
    f.write(struct.pack("50d", p["x0"], p["x1"], p["y0"], p["y1"], p["gamma"], p["Pr"], p["Re"],
                        p.get("eps_pp", 1e-12), p.get("eps_weno", 1e-8), t, *st, *bd))


def run(exe, tmp_path, p, q, t=0.0, mixed=False, dumps=False):
    """(rhs, vhat, theta, alpha*, beta_max, limiter activations, flags) of the host run,
    and with dumps the intermediate fields {0: face, 1: vol, 2: rm, 3: grad} as
    hweno_debug_fields exports them"""
    nx, ny = p["nx"], p["ny"]
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    with open(fin, "wb") as f:
        write_header(f, p, t, mixed)
        f.write(np.ascontiguousarray(q, dtype=np.float64).tobytes())
    subprocess.check_call([exe, fin, fout])
    o = np.fromfile(fout, dtype=np.float64)
    m = nx * ny
    head = (o[:12 * m].reshape(12, ny, nx), o[12 * m:20 * m].reshape(8, ny, nx), o[20 * m:22 * m].reshape(2, ny, nx),
            *o[22 * m:22 * m + 4])
    if not dumps:
        return head
    fields, at = {}, 22 * m + 4
    for k, n in ((0, 48), (1, 36), (2, 18), (3, 126)):
        fields[k] = o[at:at + n * m].reshape(n, ny, nx)
        at += n * m
    return head + (fields,)


def open_rough():
    case, q = I.random_rough(40, 36, seed=9, bc=("inflow", "outflow", "symmetry", "outflow"), Re=200.0)
    case.inflow = ((tuple(q[:4, 18, 0]), tuple(q[:4, 5, 0])), None, None, None)
    case.band = ((0.5, 0.15), None, None, None)
    return case, q


def y_jet():
    case, q = I.random_smooth(33, 29, seed=10, bc=("outflow", "outflow", "inflow", "outflow"))
    case.inflow = (None, None, (I.conserved(1.2, 0.1, 0.8, 1.5, case.gamma), I.conserved(1.0, 0.0, 0.2, 1.0, case.gamma)),
                   None)
    case.band = (None, None, (0.5, 0.2), None)
    return case, q


CASES = {
    "smooth_periodic_64": lambda: I.smooth_periodic(64),
    "rough_periodic_40x36": lambda: I.random_rough(40, 36, seed=1),
    "smooth_walls_37x29": lambda: I.random_smooth(37, 29, seed=2, bc=("noslip", "slip", "symmetry", "noslip")),
    "rough_walls_45x21": lambda: I.random_rough(45, 21, seed=3, bc=("noslip", "noslip", "noslip", "symmetry")),
    "shock_tube_64x32": lambda: I.shock_tube(64, 32),
    "taylor_green_48": lambda: I.taylor_green(48, 0.4, 300.0, 1 / 1.4, rho_pert=1e-2),
    "minimum_grid_4x4": lambda: I.random_smooth(4, 4, seed=5),
    "thin_grid_5x70": lambda: I.random_smooth(5, 70, seed=6, bc=("slip", "slip", "periodic", "periodic")),
    "open_rough_40x36": open_rough,
    "y_jet_33x29": y_jet,
    "outflow_box_37x29": lambda: I.random_smooth(37, 29, seed=11, bc=("outflow",) * 4),
    "mach2000_32x16": lambda: I.mach2000(32, 16),
    "sedov_24": lambda: I.sedov_2d(24),
    "open_shock_tube_32x16": lambda: I.open_shock_tube(32, 16),
}


def check(exe, tmp_path, case, q, t=0.0, **kw):
    p = dict(case.params(), **kw)
    rhs, vhat, theta, alpha, beta, pp, flags = run(exe, tmp_path, p, q, t)
    o = O.residual(O.make_cfg(**p, time=t), q, dumps=True)
    tol = res_tol(case, q)
    assert rel_linf(rhs, o["rhs"], flux_scale(case, q)) <= tol
    assert rel_linf(vhat, o["vhat"], state_scale(q)) <= tol
    # theta and the wave-speed bounds come from the same traces: the same conditioning
    assert np.abs(theta - o["theta"]).max() <= max(1e-13, tol)
    assert abs(alpha - o["diag"][0]) <= max(1e-13, tol) * o["diag"][0]
    assert abs(beta - o["diag"][1]) <= max(1e-12, tol) * o["diag"][1]
    assert flags == 0
    return rhs, o


@pytest.mark.parametrize("scheme", ["gr", "dr"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_residual_matches_the_oracle(exe, tmp_path, name, scheme):
    case, q = CASES[name]()
    check(exe, tmp_path, case, q, scheme=scheme)


@pytest.mark.parametrize("name", ["open_rough_40x36", "sedov_24", "rough_walls_45x21"])
def test_linear_gradient_ablation(exe, tmp_path, name):
    case, q = CASES[name]()
    check(exe, tmp_path, case, q, linear_grad=True)


@pytest.mark.parametrize("scheme", ["gr", "dr"])
def test_manufactured_source(exe, tmp_path, scheme):
    """Example 5.2's source at t = 0.03, on the unit square and on a shifted domain"""
    t = 0.03
    case, q = I.manufactured(24, t)
    check(exe, tmp_path, case, q, t, scheme=scheme)
    case = I.Case("manufactured_shifted_20", 20, 20, 0.3, 1.3, -0.4, 0.6, 1.4, 0.72, 100.0, source=1)
    q = I.cell_moments(case, lambda x, y: I.manufactured_prim(x, y, t, case.gamma))
    check(exe, tmp_path, case, q, t, scheme=scheme)


def test_limiter_engaged(exe, tmp_path):
    """near-vacuum colliding streams: the limited cells and theta are the oracle's, and
    cells whose 9x9 dependency square holds no limited cell match to the conditioning
    bound (the PP wave-speed bound makes the limited cells' residual ill-conditioned)"""
    case, q = I.colliding_streams(48, seed=3)
    p = case.params()
    rhs, vhat, theta, alpha, beta, pp, flags = run(exe, tmp_path, p, q)
    o = O.residual(O.make_cfg(**p), q, dumps=True)
    limited = (o["theta"][0] < 1) | (o["theta"][1] < 1)
    assert limited.any() and np.array_equal((theta[0] < 1) | (theta[1] < 1), limited)
    near = limited.copy()
    for dj in range(-4, 5):
        for di in range(-4, 5):
            near |= np.roll(np.roll(limited, dj, 0), di, 1)
    tol = res_tol(case, q)
    assert rel_linf(rhs, o["rhs"], flux_scale(case, q), ~near) <= tol
    assert rel_linf(vhat, o["vhat"], state_scale(q)) <= tol
    assert np.abs(theta - o["theta"]).max() <= tol
    assert pp == limited.sum()


@pytest.mark.parametrize("kernels", ["separate", "tiles"])
@pytest.mark.parametrize("linear_grad", [False, True])
@pytest.mark.parametrize("name", ["smooth_periodic_64", "rough_walls_45x21", "shock_tube_64x32", "open_rough_40x36",
                                  "y_jet_33x29", "thin_grid_5x70"])
def test_mixed_path(exe, tmp_path, name, linear_grad, kernels):
    """the mixed path's FP32 bodies on the hi/lo split of the ghost-filled state: within
    the mixed path's bounds of the FP64 oracle (1e-5 of the flux scale, 1e-6 of the state
    for the modified moments), with inflow ghosts holding the split of their state; with
    the separate kernels, or as a handle runs them (the gradients as k_grad_tma_mixed
    stages them, the fluxes and balances as k_flux_asm_mixed's tiles, each tile's shared
    memory starting as NaN)"""
    case, q = CASES[name]()
    p = dict(case.params(), linear_grad=linear_grad)
    rhs, vhat, theta, alpha, beta, pp, flags = run(exe, tmp_path, p, q, mixed=1 if kernels == "separate" else 3)
    o = O.residual(O.make_cfg(**p), q)
    assert rel_linf(rhs, o["rhs"], flux_scale(case, q)) <= 1e-5
    assert rel_linf(vhat, o["vhat"], state_scale(q)) <= 1e-6
    assert flags == 0


def test_mixed_path_conserves_to_fp64_roundoff(exe, tmp_path):
    """the mixed path differences FP64 face fluxes: a periodic average residual still sums
    to FP64 round-off"""
    case, q = I.random_rough(40, 36, seed=12)
    rhs = run(exe, tmp_path, case.params(), q, mixed=True)[0]
    for v in range(4):
        assert abs(rhs[v].sum()) <= 1e-13 * np.abs(rhs[v]).sum()


@pytest.mark.parametrize("name", ["rough_walls_45x21", "open_rough_40x36", "y_jet_33x29"])
def test_intermediate_fields(exe, tmp_path, name):
    """traces, volume values, weak moments and gradients as hweno_debug_fields exports
    them, against the oracle's, at the GPU parity test's bounds"""
    case, q = CASES[name]()
    *head, fields = run(exe, tmp_path, case.params(), q, dumps=True)
    o = O.residual(O.make_cfg(**case.params()), q, dumps=True)
    assert rel_linf(fields[0], o["face"], state_scale(q)) <= 1e-12
    assert rel_linf(fields[1], o["vol"], state_scale(q)) <= 1e-12
    assert rel_linf(fields[2], o["rm"]) <= 1e-12
    assert rel_linf(fields[3], o["grad"]) <= 1e-12
    assert np.abs(head[2] - o["theta"]).max() <= 1e-13
