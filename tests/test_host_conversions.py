"""The mixed path's conversions between float values and their FP64 planes are integer
operations (widen_f, narrow_exact, narrow_trunc in hweno_state.cuh).  They run here on
the host against the host's own conversion instructions: every float bit pattern widened
and narrowed back, and truncation of doubles across every exponent (tests/host/
conversions_host.cc)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_conversions_exhaustive(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ is needed to compile the conversions for the host")
    exe = str(tmp_path / "conversions")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-frounding-math", "-I" + os.path.join(HERE, "host"),
                           "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(ROOT, "paper_2608_10569_b300", "csrc"), "-o", exe,
                           os.path.join(HERE, "host", "conversions_host.cc")])
    out = dict(line.split()[:2] for line in subprocess.check_output([exe], timeout=600).decode().splitlines())
    assert out == {"widen": "0", "round_trip": "0", "trunc": "0"}, out
