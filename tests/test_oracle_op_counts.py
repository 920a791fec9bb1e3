"""Pins of the operation-counting build of the oracle (hweno_oracle_count.cpp), whose
per-cell counts are the algorithmic work the benchmark's roofline divides by.

- A function small enough to count by hand: the limiter's theta root (Sec. 3.1), in
  both of its branches.  Quadratic branch, with eps and gamma state-free: the four
  differences d = uq - ub (4 add); a = d3 d0 - (d1^2 + d2^2)/2 (4 mul, 2 add);
  b = E d0 + rho d3 - (m d1 + n d2) - e1 d0 (5 mul, 4 add); c = E rho - (m^2 + n^2)/2
  - e1 rho (5 mul, 3 add); the discriminant b^2 - (4 a) c (3 mul, 1 add); its square
  root; q = -(b + sign(b) sqrt)/2 (1 add, 1 mul); the roots q/a and c/q (2 div):
  15 add, 18 mul, 2 div, 1 sqrt.  Linear branch (a = 0): the same a, b, c, then -c/b:
  13 add, 14 mul, 1 div.
- Linearity in the work: evaluating one reconstruction at k distinct points costs k
  times one point.
- No halo and no state dependence: the per-cell counts of the spatial operator are the
  same on an 8^2 and a 10^2 periodic grid and on different smooth states.
- A planted miscount (operand keys that drop the sign of a state-free operand, so that
  x*c and x*(-c) merge) lowers the counts by a third: each state-free constant must
  key by its full bit pattern.
- The benchmark's flop constants are these counts.
"""
import os
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_10569_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_theta_root_quadratic_branch_by_hand():
    ub = np.array([1.0, 0.3, -0.2, 2.5])
    uq = np.array([0.7, 0.9, 0.4, 0.31])
    t, c = O.op_count_theta_root(ub, uq, 1e-12, 1.4)
    assert 0.0 < t < 1.0
    assert c == {"add": 15, "mul": 18, "div": 2, "sqrt": 1, "trans": 0}


def test_theta_root_linear_branch_by_hand():
    ub = np.array([1.0, 0.3, -0.2, 2.5])
    uq = ub.copy()
    uq[3] = 0.1  # only the energy differs: the quadratic's leading coefficient is 0
    _, c = O.op_count_theta_root(ub, uq, 1e-12, 1.4)
    assert c == {"add": 13, "mul": 14, "div": 1, "sqrt": 0, "trans": 0}


def test_evaluation_count_is_linear_in_the_points():
    d = np.random.default_rng(1).normal(size=17)
    pts = [(0.1234567 * k + 0.0101, -0.3 + 0.0712345 * k) for k in range(1, 7)]
    build1, one = O.op_count_hweno(d, pts[:1])
    for k in range(2, 7):
        build, ev = O.op_count_hweno(d, pts[:k])
        assert build == build1
        assert all(ev[key] == k * one[key] for key in O.OP_KINDS)
    # with the linear weights the indicators still run (as the oracle writes the build)
    # but the weights' arithmetic does not
    build_lin, _ = O.op_count_hweno(d, pts[:1], linear=True)
    assert O.flops(build_lin) < O.flops(build1)


def counts(gen, **extra):
    case, q = gen()
    return O.algorithmic_flops(O.make_cfg(**dict(case.params(), **extra)), q)


def test_counts_per_cell_have_no_halo_and_no_state_dependence():
    a = counts(lambda: I.random_smooth(8, 8, seed=3))
    assert counts(lambda: I.random_smooth(10, 10, seed=3)) == a
    assert counts(lambda: I.random_smooth(8, 8, seed=4)) == a
    assert counts(lambda: I.taylor_green(8, 0.4, 300.0, 1 / 1.4, rho_pert=1e-2)) == a
    assert all(v > 0 for v in a.values())


def planted_counter(tmp_path):
    """a copy of the counting build whose operand keys drop the sign of a state-free
    operand, so that x*c and x*(-c) count as one computation"""
    import ctypes
    import shutil
    import subprocess
    src = open(O._CNT_SRC).read()
    old = "    memcpy(&b, &a.v, sizeof(b));\n    return b;\n"
    assert src.count(old) == 1
    d = tmp_path / "plant"
    d.mkdir()
    (d / "hweno_oracle_count.cpp").write_text(src.replace(old, old.replace("return b;", "return b << 1;")))
    for f in ("hweno_oracle.c", "oracle_tables.h"):
        shutil.copy(os.path.join(os.path.dirname(O._SRC), f), d / f)
    lib = d / "libplant.so"
    subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c++17", "-fpermissive",
                           "-w", "-o", str(lib), str(d / "hweno_oracle_count.cpp"), "-lm"])
    return lib


def test_planted_sign_merge_changes_the_count(tmp_path, monkeypatch):
    case, q = I.random_smooth(8, 8, seed=3)
    cfg = O.make_cfg(**case.params())
    good = O.algorithmic_flops(cfg, q)
    monkeypatch.setattr(O, "_CNT_LIB", str(planted_counter(tmp_path)))
    monkeypatch.setattr(O, "_cnt", None)
    monkeypatch.setattr(O, "build", lambda force=False: O._LIB)
    bad = O.algorithmic_flops(cfg, q)
    assert bad["traces"] < 0.8 * good["traces"] and bad["gradients"] < 0.8 * good["gradients"]


def bench_module():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_bench_constants_are_the_oracle_counts():
    b = bench_module()
    gr = counts(lambda: I.random_smooth(8, 8, seed=3))
    dr = counts(lambda: I.random_smooth(8, 8, seed=3), scheme="dr")
    assert b.ALG_FLOPS["gr"] == pytest.approx(gr, rel=0, abs=1e-9)
    assert b.ALG_FLOPS["dr"] == pytest.approx(dr, rel=0, abs=1e-9)
