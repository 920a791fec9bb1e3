"""The 1D solver's GPU tests run on the CPU, with the kernel's own code standing in for
the GPU: `advance1d`, `step1d` and `residual1d` of the binding are replaced, for the
duration of each test, by calls of `k_solve` compiled for the host (`host/kernel1d_host.cc`
through `test_host1d`), and CUDA tensors by host copies.  Every assertion of
`test_zzz_gpu_1d.py` (step counts, restarts, limiter activations, tolerances) then meets
an arithmetic other than the oracle's before it meets the GPU's.
"""
import inspect

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import test_host1d as H  # noqa: E402
import test_zzz_gpu_1d as G  # noqa: E402
from paper_2608_10569_b300 import hweno  # noqa: E402

exe = H.exe  # the host build of the kernel (module fixture)


def _cases():
    out = []
    for name, fn in inspect.getmembers(G, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        combos = [{}]
        for m in getattr(fn, "pytestmark", []):
            if m.name == "parametrize":
                keys = [k.strip() for k in m.args[0].split(",")]
                combos = [dict(c, **dict(zip(keys, v if len(keys) > 1 else (v,)))) for c in combos for v in m.args[1]]
        out += [(name, c) for c in combos]
    return out


@pytest.mark.parametrize("name,kwargs", _cases(), ids=lambda x: str(x) if isinstance(x, str) else "-".join(map(str, x.values())))
def test_gpu_test_on_the_host_kernel(exe, tmp_path, monkeypatch, name, kwargs):
    def advance1d(params_list, states, t0, t_end, max_steps=2 ** 31 - 1, stream=None):
        if len(states) != len(params_list):
            raise ValueError("one state per problem")
        out = []
        for p, st in zip(params_list, states):
            q, o = H.run(exe, tmp_path, p, st.numpy(), 0, t0, t_end, max_steps)
            st.copy_(torch.from_numpy(q))
            out.append({"t": o[0], "steps": int(o[1]), "rejections": int(o[2]), "status": int(o[3]),
                        "pp_active": int(o[4])})
        return out

    def step1d(params, state, t, dt=0.0, stream=None):
        q, o = H.run(exe, tmp_path, params, state.numpy(), 1, t, np.inf, 1, dt)
        state.copy_(torch.from_numpy(q))
        return {"dt": o[0], "rejections": int(o[2]), "status": int(o[3]), "pp_active": int(o[4])}

    def residual1d(params, state, t=0.0, stream=None):
        rhs, vh, _ = H.run(exe, tmp_path, params, state.numpy(), 2, t0=t)
        return torch.from_numpy(rhs.copy()), torch.from_numpy(vh.copy())

    monkeypatch.setattr(hweno, "advance1d", advance1d)
    monkeypatch.setattr(hweno, "step1d", step1d)
    monkeypatch.setattr(hweno, "residual1d", residual1d)
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self.clone())
    getattr(G, name)(**kwargs)
