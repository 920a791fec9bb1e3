"""The open-face GPU tests run on the CPU, with the kernels' own code standing in for the
GPU: for the duration of each test, `hweno.Solver` and `hweno.Batch` are replaced by
stand-ins whose residuals come from `host/residual2d_host.cc` and whose steps (forced or
by the rule, with the restart rule) come from `host/step2d_host.cc`, and CUDA tensors by
host copies.  The assertions of `test_zzy_gpu_open.py` then meet an arithmetic other
than the oracle's before they meet the GPU's.  Tests of `hweno_residual_noalloc` and
of the adjoint have no stand-in and are not run here.
"""
import inspect

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import test_host_residual2d as R  # noqa: E402
import test_host_step2d as S  # noqa: E402
import test_zzy_gpu_open as G  # noqa: E402
from paper_2608_10569_b300 import hweno  # noqa: E402

NOT_HERE = {"test_noalloc_with_open_faces", "test_adjoint_dot_products_with_open_faces",
            "test_adjoint_with_the_linear_gradient_ablation"}


@pytest.fixture(scope="module")
def exes(tmp_path_factory):
    import os
    import shutil
    import subprocess
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ is needed to compile the device code for the host")
    d = tmp_path_factory.mktemp("open_rehearsal")
    out = {}
    for name in ("residual2d_host", "step2d_host"):
        exe = str(d / name)
        cmd = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fno-strict-aliasing", "-I" + os.path.join(R.HERE, "host"),
               "-I" + os.path.join(R.ROOT, "include"), "-I" + R.CSRC, "-o", exe,
               os.path.join(R.HERE, "host", name + ".cc")]
        subprocess.check_call(cmd)
        out[name] = exe
    return out


def _cases():
    out = []
    for name, fn in inspect.getmembers(G, inspect.isfunction):
        if not name.startswith("test_") or name in NOT_HERE:
            continue
        combos = [{}]
        for m in getattr(fn, "pytestmark", []):
            if m.name == "parametrize":
                keys = [k.strip() for k in m.args[0].split(",")]
                combos = [dict(c, **dict(zip(keys, v if len(keys) > 1 else (v,)))) for c in combos for v in m.args[1]]
        out += [(name, c) for c in combos]
    return out


class _Case:
    """the parameters of a solver as the harnesses read them"""

    def __init__(self, params):
        self._p = dict(params)
        self.gamma, self.nx, self.ny = self._p["gamma"], self._p["nx"], self._p["ny"]

    def params(self):
        return dict(self._p)


def _solver_class(exes, tmp_path):
    class Solver:
        def __init__(self, params, precision="fp64", stream=None):
            self.p = dict(params)
            self.mixed = precision == "mixed"
            self.t, self.steps, self.rejected, self.dt_last = 0.0, 0, 0, 0.0
            self.d = (0.0, 0.0)

        def set_state(self, q):
            self.q = np.array(q.numpy() if torch.is_tensor(q) else q, dtype=np.float64)

        def residual(self):
            r = R.run(exes["residual2d_host"], tmp_path, self.p, self.q, self.t, mixed=self.mixed, dumps=True)
            self.fields = dict(r[7])
            self.fields[4] = r[2]
            self.d = (r[3], r[4])
            return torch.from_numpy(r[0].copy()), torch.from_numpy(r[1].copy())

        def debug_fields(self, which):
            return torch.from_numpy(self.fields[which].copy())

        def step(self, dt=0.0):
            q, status, log = S.steps(exes["step2d_host"], tmp_path, _Case(self.p), self.q, 1, t=self.t, dt=dt,
                                     mixed=self.mixed)
            if status != 0:
                self.rejected += log[-1][1]
                raise hweno.HwenoError(status, "inadmissible")
            (dt_used, rej), = log
            self.q, self.t, self.dt_last = q, self.t + dt_used, dt_used
            self.steps += 1
            self.rejected += rej
            return dt_used, rej

        def diag(self):
            return {"t": self.t, "dt_last": self.dt_last, "alpha_star": self.d[0], "beta_max": self.d[1],
                    "steps": self.steps, "rejected": self.rejected}

        def get_state(self, out=None):
            if out is not None:
                out[...] = self.q
                return out
            return torch.from_numpy(self.q.copy())

        def close(self):
            pass

    class Batch:
        def __init__(self, plist, precision="mixed", stream=None):
            self.cases = [Solver(p, precision) for p in plist]

        def step(self, n=1):
            for c in self.cases:
                for _ in range(n):
                    c.step()

        def close(self):
            pass

    return Solver, Batch


@pytest.mark.parametrize("name,kwargs", _cases(), ids=lambda x: str(x) if isinstance(x, str) else "-".join(map(str, x.values())))
def test_gpu_test_on_the_host_kernels(exes, tmp_path, monkeypatch, name, kwargs):
    solver, batch = _solver_class(exes, tmp_path)
    monkeypatch.setattr(hweno, "Solver", solver)
    monkeypatch.setattr(hweno, "Batch", batch)
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self.clone())
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: None)
    getattr(G, name)(**kwargs)
