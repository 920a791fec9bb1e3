"""The 2D ghost-cell rules of the CUDA path (Remark 4.1; `csrc/hweno_state.cuh`, the
code the ghost kernels run) compiled for the host with `host/shim.h` and run over whole
states, against the oracle's ghost fill: every padded cell, corners included, must be
identical, for every kind of face (periodic, the three walls, inflow with a band and
outflow) and their combinations.  The 24 float planes of the mixed path's hi/lo split,
filled by the same rules, must hold the split of the FP64 ghost values, which a numpy
restatement of the split gives independently.
"""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_10569_b300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
# out-of-bounds reads and writes of the kernel's index arithmetic, and undefined
# behaviour, abort the run where the compiler has the sanitizers
SANITIZE = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-g"]
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2608_10569_b300", "csrc")
BC = {"periodic": 0, "noslip": 1, "symmetry": 2, "slip": 3, "inflow": 4, "outflow": 5}
G = 4


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ is needed to compile the device code for the host")
    out = str(tmp_path_factory.mktemp("ghost2d") / "ghost2d_host")
    cmd = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I" + os.path.join(HERE, "host"),
           "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-o", out, os.path.join(HERE, "host", "ghost2d_host.cc")]
    if subprocess.run(cmd + SANITIZE, capture_output=True).returncode != 0:
        subprocess.check_call(cmd)
    return out


def run(exe, tmp_path, p, q):
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
        f.write(struct.pack("6i", nx, ny, *[BC[b] for b in p["bc"]]))
        f.write(struct.pack("44d", p["x0"], p["x1"], p["y0"], p["y1"], *st, *bd))
        f.write(np.ascontiguousarray(q, dtype=np.float64).tobytes())
    subprocess.check_call([exe, fin, fout])
    raw = open(fout, "rb").read()
    nd = 12 * (ny + 2 * G) * (nx + 2 * G)
    dbl = np.frombuffer(raw[:8 * nd], dtype=np.float64).reshape(12, ny + 2 * G, nx + 2 * G)
    flt = np.frombuffer(raw[8 * nd:], dtype=np.float32).reshape(24, ny + 2 * G, nx + 2 * G)
    return dbl, flt


def split(x):
    """hi: x with its mantissa truncated to 24 significant bits; lo: the exact remainder
    x - hi truncated the same way (values of normal float range)"""
    mask = np.uint64(~((1 << 29) - 1) & 0xFFFFFFFFFFFFFFFF)
    hi = (x.view(np.uint64) & mask).view(np.float64)
    lo = ((x - hi).view(np.uint64) & mask).view(np.float64)
    return hi.astype(np.float32), lo.astype(np.float32)


A = I.conserved(1.5, 0.6, 0.1, 3.0, 1.4)
B = I.conserved(1.1, 0.2, -0.1, 2.5, 1.4)
C = I.conserved(0.9, 0.0, -0.3, 2.2, 1.4)
D = I.conserved(0.7, -0.4, 0.5, 1.2, 1.4)

FACES = {
    "inflow_outflow_symmetry_inflow": (("inflow", "outflow", "symmetry", "inflow"),
                                       ((A, B), None, None, (C, C)), ((0.5, 0.2), None, None, None)),
    "outflow_everywhere": (("outflow",) * 4, None, None),
    "periodic_x_inflow_y": (("periodic", "periodic", "inflow", "outflow"),
                            (None, None, (A, D), None), (None, None, (0.3, 0.0), None)),
    "noslip_inflow_outflow_slip": (("noslip", "inflow", "outflow", "slip"),
                                   (None, (B, C), None, None), (None, (0.45, 0.125), None, None)),
    "inflow_everywhere": (("inflow",) * 4, ((A, B), (B, C), (C, D), (D, A)),
                          ((0.5, 0.25), (0.2, 0.1), (0.75, 0.2), (0.5, 0.5))),
    "inflow_x_noslip_y": (("inflow", "symmetry", "noslip", "noslip"),
                          ((A, D), None, None, None), ((0.6, 0.3), None, None, None)),
    "walls": (("noslip", "symmetry", "slip", "noslip"), None, None),
    "periodic": (("periodic",) * 4, None, None),
    "periodic_y_open_x": (("inflow", "outflow", "periodic", "periodic"),
                          ((C, A), None, None, None), ((0.5, 0.1), None, None, None)),
}


@pytest.mark.parametrize("shape", [(13, 10), (4, 4), (5, 9)])
@pytest.mark.parametrize("name", sorted(FACES))
def test_ghost_fill_matches_the_oracle(exe, tmp_path, name, shape):
    bc, inflow, band = FACES[name]
    nx, ny = shape
    case, q = I.random_smooth(nx, ny, seed=nx * ny, bc=("symmetry",) * 4)
    p = dict(case.params(), bc=bc, inflow=inflow, band=band, x0=-0.3, x1=0.9, y0=0.1, y1=1.1)
    dbl, flt = run(exe, tmp_path, p, q)
    ref = O.fill_ghosts(O.make_cfg(**p), q)
    assert np.array_equal(dbl, ref)
    hi, lo = split(ref)
    assert np.array_equal(flt[:12], hi) and np.array_equal(flt[12:], lo)


@pytest.mark.parametrize("make", [lambda: I.sedov_2d(12), lambda: I.mach2000(24, 12)])
def test_benchmark_setups(exe, tmp_path, make):
    """Examples 5.7 and 5.9: the corner blast and the jet"""
    case, q = make()
    p = case.params()
    dbl, flt = run(exe, tmp_path, p, q)
    ref = O.fill_ghosts(O.make_cfg(**p), q)
    assert np.array_equal(dbl, ref)
    hi, lo = split(ref)
    assert np.array_equal(flt[:12], hi) and np.array_equal(flt[12:], lo)


def test_band_edges_follow_the_coordinates(exe, tmp_path):
    """band edges between cell centres and a zero half width (state B alone), on a
    domain whose centres are not dyadic"""
    nx, ny = 7, 11
    case, q = I.random_smooth(nx, ny, seed=3, bc=("symmetry",) * 4)
    for band in ((0.35, 0.1), (0.35, 0.0), (-5.0, 1.0), (0.5, 10.0)):
        p = dict(case.params(), bc=("inflow", "inflow", "inflow", "inflow"), x0=0.1, x1=0.8, y0=-0.2, y1=0.9,
                 inflow=((A, B), (B, A), (C, D), (D, C)), band=(band,) * 4)
        dbl, _ = run(exe, tmp_path, p, q)
        assert np.array_equal(dbl, O.fill_ghosts(O.make_cfg(**p), q)), band
