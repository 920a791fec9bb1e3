"""The discrete adjoints of the spatial operator (Eq. (3.2), with the PP limiter and the
modified moments) and of one SSP-RK3 step at a fixed dt, run on the host, against the
oracle's forward-mode (dual-number) tangents.

`host/residual_adjoint_host.cc` compiles the CUDA path's recording forward, its stage
update and its reverse kernels (`hweno_adjoint.cuh`) as plain C++ with `host/shim.h`,
calls each over the index range of its launch in the order of hweno_adjoint_residual or
hweno_adjoint_step, and starts every plane that the sequence does not clear or seed as
NaN, under AddressSanitizer and UBSan where the compiler has them.  For seeds (rbar,
mbar) and a tangent (v, dmu), <(rbar, mbar), J (v, dmu)> from the oracle's tangent must
equal <xbar, v> + mubar dmu from the sweep, and <lam', J_step v> must equal <lam, v> for
the step: the GPU adjoint tests' dot products, with the same 1e-10, here without the
GPU's arithmetic and thread interleaving (which those tests cover).  The recording
forward's residual and step must also be the oracle's.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_10569_b300 import inputs as I
from parity_tools import flux_scale, rel_linf, res_tol
from test_host_residual2d import CSRC, HERE, ROOT, SANITIZE, write_header


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ is needed to compile the device code for the host")
    out = str(tmp_path_factory.mktemp("residual_adjoint") / "residual_adjoint_host")
    cmd = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fno-strict-aliasing", "-I" + os.path.join(HERE, "host"),
           "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-o", out,
           os.path.join(HERE, "host", "residual_adjoint_host.cc")]
    if subprocess.run(cmd + SANITIZE, capture_output=True).returncode != 0:
        subprocess.check_call(cmd)
    return out


def _run(exe, tmp_path, p, mode, dt, arrays):
    nx, ny = p["nx"], p["ny"]
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    with open(fin, "wb") as f:
        write_header(f, p)
        f.write(struct.pack("=id", mode, dt))
        for a in arrays:
            f.write(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    subprocess.check_call([exe, fin, fout])
    o = np.fromfile(fout, dtype=np.float64)
    m = nx * ny
    return o[:12 * m].reshape(12, ny, nx), o[12 * m], o[12 * m + 1:24 * m + 1].reshape(12, ny, nx)


def sweep(exe, tmp_path, p, q, rbar, mbar):
    """(xbar, mubar, rhs) of the host sweep"""
    return _run(exe, tmp_path, p, 0, 0.0, (q, rbar, mbar))


def step_adjoint(exe, tmp_path, p, q, dt, lam_next):
    """(lam, mubar, q_next) of the host step adjoint at the fixed dt"""
    return _run(exe, tmp_path, p, 1, dt, (q, lam_next))


def open_jet():
    case, q = I.random_smooth(18, 14, seed=38, bc=("inflow", "outflow", "symmetry", "outflow"))
    case.inflow = ((tuple(q[:4, 7, 0]), tuple(q[:4, 2, 0])), None, None, None)
    case.band = ((0.5, 0.2), None, None, None)
    return case, q, {}


CASES = {
    "walls_16": lambda: I.random_smooth(16, 16, seed=35, bc=("noslip", "noslip", "noslip", "symmetry")) + ({},),
    "periodic_taylor_green_16": lambda: I.taylor_green(16, 0.5, 300.0, 1 / (1.4 * 0.09), rho_pert=1e-3, seed=36)
    + ({},),
    "ragged_slip_13x9": lambda: I.random_smooth(13, 9, seed=39, bc=("slip", "symmetry", "periodic", "periodic"))
    + ({},),
    "linear_gradients_walls_15x12": lambda: I.random_smooth(15, 12, seed=40, bc=("noslip", "slip", "noslip",
                                                                                  "symmetry")) + ({"linear_grad": True},),
    # eps_PP raised so that the limiter acts in many cells of a well-conditioned state
    "limited_density": lambda: I.random_smooth(16, 16, seed=37, bc=("noslip", "noslip", "noslip", "symmetry"))
    + ({"eps_pp": 0.85},),
    "limited_pressure": lambda: I.random_smooth(16, 16, seed=35, bc=("noslip", "noslip", "noslip", "symmetry"))
    + ({"eps_pp": 0.9},),
    "open_jet_18x14": open_jet,
}


def _rel(a, b):
    return abs(a - b) / max(abs(a), abs(b))


@pytest.mark.parametrize("name", sorted(CASES))
def test_sweep_is_the_transpose_of_the_oracle_tangent(exe, tmp_path, name):
    case, q, extra = CASES[name]()
    p = dict(case.params(), **extra)
    cfg = O.make_cfg(**p)
    rng = np.random.default_rng(81)
    v = rng.normal(size=q.shape) * np.abs(q).reshape(12, -1).max(1)[:, None, None]
    rbar = rng.normal(size=q.shape)
    mbar = rng.normal(size=(8,) + q.shape[1:])
    xbar, mub, rhs = sweep(exe, tmp_path, p, q, rbar, mbar)
    o = O.residual(cfg, q, dumps=True)
    assert rel_linf(rhs, o["rhs"], flux_scale(case, q)) <= res_tol(case, q)
    if "eps_pp" in extra:
        assert (o["theta"] < 1).sum() >= 5
    t = O.residual_jvp(cfg, q, v)
    tm = O.residual_jvp(cfg, q, None, dmu=1.0)
    lhs = (rbar * t["rhs_dot"]).sum() + (mbar * t["vhat_dot"]).sum()
    assert _rel(lhs, (xbar * v).sum()) <= 1e-10, (lhs, (xbar * v).sum())
    lhs_mu = (rbar * tm["rhs_dot"]).sum() + (mbar * tm["vhat_dot"]).sum()
    assert _rel(lhs_mu, mub) <= 1e-10, (lhs_mu, mub)


def test_a_wrong_seed_is_seen(exe, tmp_path):
    """the dot product separates: one seed value changed moves <xbar, v> well past 1e-10"""
    case, q, _ = CASES["walls_16"]()
    p = case.params()
    rng = np.random.default_rng(82)
    v = rng.normal(size=q.shape) * np.abs(q).reshape(12, -1).max(1)[:, None, None]
    rbar = rng.normal(size=q.shape)
    mbar = rng.normal(size=(8,) + q.shape[1:])
    t = O.residual_jvp(O.make_cfg(**p), q, v)
    lhs = (rbar * t["rhs_dot"]).sum() + (mbar * t["vhat_dot"]).sum()
    r2 = rbar.copy()
    r2[5, 7, 3] += 1e-3
    xbar, _, _ = sweep(exe, tmp_path, p, q, r2, mbar)
    assert _rel(lhs, (xbar * v).sum()) > 1e-8


@pytest.mark.parametrize("name", sorted(CASES))
def test_step_adjoint_is_the_transpose_of_the_oracle_tangent(exe, tmp_path, name):
    case, q, extra = CASES[name]()
    p = dict(case.params(), **extra)
    cfg = O.make_cfg(**p)
    dt = 0.25 * O.step(cfg, q)[1]["dt"]
    rng = np.random.default_rng(83)
    v = rng.normal(size=q.shape) * np.abs(q).reshape(12, -1).max(1)[:, None, None]
    lam_next = rng.normal(size=q.shape)
    lam, mub, q_next = step_adjoint(exe, tmp_path, p, q, dt, lam_next)
    q_or, t, st = O.step_jvp(cfg, q, v, dt)
    assert st["status"] == 0 and st["rejections"] == 0
    scale = np.abs(q[:4]).reshape(4, -1).max(1)
    err = max(np.abs(q_next[k] - q_or[k]).max() / max(np.abs(q_or[k]).max(), scale[k % 4]) for k in range(12))
    assert err <= 1e-12, err
    assert _rel((lam_next * t).sum(), (lam * v).sum()) <= 1e-10
    _, tm, _ = O.step_jvp(cfg, q, np.zeros_like(q), dt, dmu=1.0)
    assert _rel((lam_next * tm).sum(), mub) <= 1e-10
