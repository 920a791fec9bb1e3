"""The adjoint of the gradient reconstruction with the linear weights (Remark 3.1's
ablation: `ka_grad<true>`), compiled for the host with `host/shim.h`, against its
forward (`grad_body` with the linear weights): that map is linear in the 17 stencil data
of each field, so <lambda, F(rm)> must equal the reverse's contributions dotted with the
stencil data, to rounding, on any data.  `host/grad_adjoint_host.cc` computes both sums.
"""
import os
import shutil
import subprocess

import pytest

from test_host_residual2d import CSRC, HERE, ROOT, SANITIZE


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ is needed to compile the device code for the host")
    out = str(tmp_path_factory.mktemp("grad_adjoint") / "grad_adjoint_host")
    cmd = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fno-strict-aliasing", "-I" + os.path.join(HERE, "host"),
           "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-o", out, os.path.join(HERE, "host", "grad_adjoint_host.cc")]
    if subprocess.run(cmd + SANITIZE, capture_output=True).returncode != 0:
        subprocess.check_call(cmd)
    return out


@pytest.mark.parametrize("nx,ny,seed", [(13, 9, 1), (4, 4, 2), (21, 6, 3)])
def test_linear_gradient_adjoint_is_the_transpose(exe, nx, ny, seed):
    lhs, rhs, scale = map(float, subprocess.check_output([exe, str(nx), str(ny), str(seed)]).split())
    assert abs(lhs - rhs) <= 1e-13 * scale
    assert scale > 0
