"""The adjoint of the ghost fill (`ka_ghost_y`, `ka_ghost_x` in `csrc/hweno_adjoint.cuh`),
compiled for the host with `host/shim.h` and called once per thread index, against the
forward ghost passes: with the inflow states at zero the ghost fill G is linear, so for
any state q and any padded adjoint field lambda, <G q, lambda> over the padded planes
equals <q, G^T lambda> over the interior.  This holds for every kind of face (a mirror
returns the ghost's adjoint with the ghost's sign, an outflow ghost's goes to the edge
cell, an inflow ghost's is dropped) and for the corners, where the two passes compose.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_10569_b300 import inputs as I
from test_host_ghost2d import BC, FACES, G

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2608_10569_b300", "csrc")
SANITIZE = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-g"]


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ is needed to compile the device code for the host")
    out = str(tmp_path_factory.mktemp("ghost_adjoint") / "ghost_adjoint_host")
    cmd = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fno-strict-aliasing", "-I" + os.path.join(HERE, "host"),
           "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-o", out, os.path.join(HERE, "host", "ghost_adjoint_host.cc")]
    if subprocess.run(cmd + SANITIZE, capture_output=True).returncode != 0:
        subprocess.check_call(cmd)
    return out


@pytest.mark.parametrize("shape", [(13, 10), (4, 4), (5, 9)])
@pytest.mark.parametrize("name", sorted(FACES))
def test_ghost_adjoint_is_the_transpose(exe, tmp_path, name, shape):
    bc, inflow, band = FACES[name]
    nx, ny = shape
    case, q = I.random_smooth(nx, ny, seed=nx * ny + 1, bc=("symmetry",) * 4)
    lam = np.random.default_rng(nx + 7 * ny).standard_normal((12, ny + 2 * G, nx + 2 * G))
    bd = []
    for k in range(4):
        bd += list(band[k]) if band and band[k] is not None else [0.0, 0.0]
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    with open(fin, "wb") as f:
        f.write(struct.pack("6i", nx, ny, *[BC[b] for b in bc]))
        f.write(struct.pack("12d", -0.3, 0.9, 0.1, 1.1, *bd))
        f.write(np.ascontiguousarray(q).tobytes())
        f.write(np.ascontiguousarray(lam).tobytes())
    subprocess.check_call([exe, fin, fout])
    out = np.fromfile(fout)
    m = 12 * (ny + 2 * G) * (nx + 2 * G)
    gq = out[:m].reshape(12, ny + 2 * G, nx + 2 * G)
    adj = out[m:].reshape(12, ny, nx)
    # the forward part is the oracle's ghost fill with the inflow states at zero
    zero = tuple(((0.0,) * 4, (0.0,) * 4) if (inflow and inflow[k] is not None) else None for k in range(4))
    p = dict(case.params(), bc=bc, inflow=zero, band=band, x0=-0.3, x1=0.9, y0=0.1, y1=1.1)
    assert np.array_equal(gq, O.fill_ghosts(O.make_cfg(**p), q))
    lhs = float((gq * lam).sum())
    rhs = float((q * adj).sum())
    assert abs(lhs - rhs) <= 1e-13 * float((np.abs(gq) * np.abs(lam)).sum())
