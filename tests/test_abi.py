"""Host-side checks of the C ABI: the library loads, exports every entry point
that include/hweno.h declares, and validates configurations without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in ("hweno.h", "hweno1d.h"):
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(hweno1?d?_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2608_10569_b300 import build, hweno
    build.build()
    return hweno.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_2608_10569_b300 import hweno
    bound = {n for n, _, _ in hweno.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_config_default_matches_the_paper(lib):
    from paper_2608_10569_b300 import hweno
    c = hweno.hweno_config()
    assert lib.hweno_config_default(ctypes.byref(c)) == 0
    assert (c.cfl, c.b_visc, c.eps_pp, c.eps_weno) == (0.6, 1e-3, 1e-12, 1e-8)
    assert (c.gamma, c.Pr, c.max_halvings) == (1.4, 0.72, 60)


def test_invalid_configurations_are_rejected_before_any_device_call(lib):
    from paper_2608_10569_b300 import hweno
    h = ctypes.c_void_p()
    bad = [dict(nx=3, ny=8), dict(nx=8, ny=8, bc=("periodic", "noslip", "periodic", "periodic")),
           dict(nx=8, ny=8, Re=0.0), dict(nx=8, ny=8, x1=0.0), dict(nx=8, ny=8, precision=7)]
    for kw in bad:
        c = hweno.make_config(**kw)
        if kw.get("precision") == 7:
            c.precision = 7
        rc = lib.hweno_init(ctypes.byref(c), None, ctypes.byref(h))
        assert rc == hweno.HWENO_ERR_ARG, kw
        assert h.value is None
        assert lib.hweno_last_error(None)


def test_null_handle_calls_fail_cleanly(lib):
    from paper_2608_10569_b300 import hweno
    assert lib.hweno_step(None, 0.0, None, None) == hweno.HWENO_ERR_ARG
    assert lib.hweno_residual(None, None, None, 0) == hweno.HWENO_ERR_ARG
    assert lib.hweno_launch_count(None) == 0


def test_gpu_and_oracle_tables_agree():
    """The GPU constants (float64 numpy derivation) and the oracle constants (exact
    rationals) are independent derivations of Appendix A.2's stencil maps."""
    import numpy as np
    import sys
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import gen_tables as g
    Mx = np.array([[float(x) for x in r] for r in g.p0_map()])
    Bx = np.array([[float(x) for x in r] for r in g.beta_matrix()])
    txt = open(os.path.join(ROOT, "paper_2608_10569_b300", "csrc", "hweno_stencil.h")).read()
    M = np.zeros((15, 17))
    body = txt[txt.index("hw_p0_coeffs"):txt.index("hw_beta_quartic")]
    for k, expr in re.findall(r"c\[(\d+)\] = (.*?);\n", body):
        for v, n in re.findall(r"T\(([-0-9.e]+)\) \* d\[(\d+)\]", expr):
            M[int(k), int(n)] = float(v)
    assert np.abs(M - Mx).max() <= 1e-14 * np.abs(Mx).max()
    assert np.array_equal(M != 0, Mx != 0)
    body = txt[txt.index("hw_beta_quartic"):txt.index("hw_moment_xi")]
    B = np.zeros((15, 15))
    for i, expr in re.findall(r"s \+= c\[(\d+)\] \* \((.*?)\);\n", body):
        for v, j in re.findall(r"T\(([-0-9.e]+)\) \* c\[(\d+)\]", expr):
            i_, j_ = int(i), int(j)
            if i_ == j_:
                B[i_, j_] = float(v)
            else:
                B[i_, j_] = B[j_, i_] = float(v) / 2
    assert np.abs(B - Bx).max() <= 1e-13 * np.abs(Bx).max()


def test_scheme_is_validated_before_any_device_call(lib):
    """HWENO_SCHEME_DR is accepted for FP64 handles and FP64 batches of DR cases only;
    an unknown scheme, DR with the mixed precision, a batch mixing the schemes, a mixed
    DR batch and DR in hweno_residual_noalloc are refused on the host"""
    from paper_2608_10569_b300 import hweno
    h = ctypes.c_void_p()
    for kw in (dict(scheme="dr", precision="mixed"),):
        c = hweno.make_config(8, 8, **kw)
        assert lib.hweno_init(ctypes.byref(c), None, ctypes.byref(h)) == hweno.HWENO_ERR_ARG
        assert b"FP64" in lib.hweno_last_error(None)
    c = hweno.make_config(8, 8)
    c.scheme = 2
    assert lib.hweno_init(ctypes.byref(c), None, ctypes.byref(h)) == hweno.HWENO_ERR_ARG
    cfgs = (hweno.hweno_config * 2)(hweno.make_config(8, 8), hweno.make_config(8, 8, scheme="dr"))
    b = ctypes.c_void_p()
    assert lib.hweno_batch_init(cfgs, 2, None, ctypes.byref(b)) == hweno.HWENO_ERR_ARG
    assert b.value is None and b"same scheme" in lib.hweno_last_error(None)
    cfgs = (hweno.hweno_config * 1)(hweno.make_config(8, 8, scheme="dr", precision="mixed"))
    assert lib.hweno_batch_init(cfgs, 1, None, ctypes.byref(b)) == hweno.HWENO_ERR_ARG
    assert b.value is None and b"FP64" in lib.hweno_last_error(None)
    buf = (ctypes.c_double * 12)()
    c = hweno.make_config(8, 8, scheme="dr")
    assert lib.hweno_residual_noalloc(ctypes.byref(c), buf, buf, None, None) == hweno.HWENO_ERR_ARG
    assert b"GR" in lib.hweno_last_error(None)


def test_source_is_validated_before_any_device_call(lib):
    """an unknown source term and a source in hweno_residual_noalloc (which has no
    time) are refused on the host"""
    from paper_2608_10569_b300 import hweno
    h = ctypes.c_void_p()
    c = hweno.make_config(8, 8)
    c.source = 2
    assert lib.hweno_init(ctypes.byref(c), None, ctypes.byref(h)) == hweno.HWENO_ERR_ARG
    buf = (ctypes.c_double * 12)()
    c = hweno.make_config(8, 8, source="mms52")
    assert lib.hweno_residual_noalloc(ctypes.byref(c), buf, buf, None, None) == hweno.HWENO_ERR_ARG
    assert b"source" in lib.hweno_last_error(None)


def test_1d_configurations_are_validated_before_any_device_call(lib):
    """the 1D entry points check every problem's configuration on the host: cell count,
    boundary codes and periodic pairing, scheme, source and the physical constants"""
    from paper_2608_10569_b300 import hweno
    c = hweno.make_config1d(40)
    assert (c.cfl, c.b_visc, c.eps_pp, c.eps_weno, c.gamma, c.Pr) == (0.6, 1e-3, 1e-12, 1e-8, 1.4, 0.72)
    bad = [dict(n=3), dict(n=40, bc=("periodic", "outflow")), dict(n=40, scheme=2), dict(n=40, Re=0.0),
           dict(n=40, source=3), dict(n=hweno_max_cells() + 1)]
    ptr = (ctypes.c_void_p * 1)(ctypes.c_void_p(8).value)
    for kw in bad:
        kw = dict(kw)
        scheme, source = kw.pop("scheme", "gr"), kw.pop("source", 0)
        c = hweno.make_config1d(**kw)
        c.scheme, c.source = scheme if isinstance(scheme, int) else 0, source
        rc = lib.hweno1d_advance(ctypes.byref(c), 1, ptr, 0.0, 1.0, 1, None, None)
        assert rc == hweno.HWENO_ERR_ARG, kw
        assert lib.hweno1d_last_error()


def hweno_max_cells():
    txt = open(os.path.join(ROOT, "include", "hweno1d.h")).read()
    return int(re.search(r"#define HWENO1D_MAX_CELLS (\d+)", txt).group(1))


def test_struct_mirrors_match_the_headers(tmp_path):
    """the binding's ctypes structures have the C structures' size and field offsets"""
    import shutil
    import subprocess
    from paper_2608_10569_b300 import hweno
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc is needed to compile against the headers")
    structs = {"hweno_config": hweno.hweno_config, "hweno_diag": hweno.hweno_diag,
               "hweno1d_config": hweno.hweno1d_config}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hweno.h"', '#include "hweno1d.h"',
             "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (name, name))
        for f in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f[0], name, f[0]))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = str(tmp_path / "layout")
    subprocess.check_call([cc, "-std=c99", "-I" + os.path.join(ROOT, "include"), "-o", exe, str(src)])
    seen = {}
    for line in subprocess.check_output([exe]).decode().split("\n"):
        if line:
            s, f, v = line.split()
            seen[(s, f)] = int(v)
    for name, cls in structs.items():
        assert seen[(name, "sizeof")] == ctypes.sizeof(cls), name
        for f in cls._fields_:
            assert seen[(name, f[0])] == getattr(cls, f[0]).offset, (name, f[0])


def test_open_faces_are_validated_before_any_device_call(lib):
    """inflow states need rho > 0 and p > 0 and a band half width >= 0, in a handle and in
    every case of a batch"""
    from paper_2608_10569_b300 import hweno
    h = ctypes.c_void_p()
    good = (1.0, 0.5, 0.0, 2.5)
    bad = [dict(inflow=((good, (0.0, 0.0, 0.0, 1.0)), None, None, None), band=((0.5, 0.1), None, None, None)),
           dict(inflow=((good, (1.0, 2.0, 0.0, 1.0)), None, None, None), band=((0.5, 0.1), None, None, None)),
           dict(inflow=((good, good), None, None, None), band=((0.5, -0.1), None, None, None)),
           dict(inflow=((good, (1.0, float("nan"), 0.0, 2.0)), None, None, None), band=((0.5, 0.1), None, None, None))]
    for kw in bad:
        c = hweno.make_config(8, 8, bc=("inflow", "outflow", "symmetry", "symmetry"), **kw)
        assert lib.hweno_init(ctypes.byref(c), None, ctypes.byref(h)) == hweno.HWENO_ERR_ARG, kw
        assert h.value is None
    ok = hweno.make_config(8, 8, bc=("inflow", "outflow", "symmetry", "symmetry"),
                           inflow=((good, good), None, None, None), band=((0.5, 0.1), None, None, None))
    b = ctypes.c_void_p()
    cfgs = (hweno.hweno_config * 2)(ok, hweno.make_config(8, 8, bc=("inflow", "outflow", "symmetry", "symmetry"),
                                                          **bad[0]))
    assert lib.hweno_batch_init(cfgs, 2, None, ctypes.byref(b)) == hweno.HWENO_ERR_ARG
    assert b.value is None
    assert b"inflow state" in lib.hweno_last_error(None)


def test_linear_gradient_ablation_is_validated_before_any_device_call(lib):
    """linear_grad is 0 or 1, ablates HWENO-GR only, and is the same for every case of a
    batch"""
    from paper_2608_10569_b300 import hweno
    h = ctypes.c_void_p()
    c = hweno.make_config(8, 8, linear_grad=True)
    c.linear_grad = 2
    assert lib.hweno_init(ctypes.byref(c), None, ctypes.byref(h)) == hweno.HWENO_ERR_ARG
    c = hweno.make_config(8, 8, linear_grad=True, scheme="dr")
    assert lib.hweno_init(ctypes.byref(c), None, ctypes.byref(h)) == hweno.HWENO_ERR_ARG
    assert h.value is None
    b = ctypes.c_void_p()
    cfgs = (hweno.hweno_config * 2)(hweno.make_config(8, 8, linear_grad=True), hweno.make_config(8, 8))
    assert lib.hweno_batch_init(cfgs, 2, None, ctypes.byref(b)) == hweno.HWENO_ERR_ARG
    assert b.value is None and b"linear_grad" in lib.hweno_last_error(None)


def test_binding_refuses_buffers_of_the_wrong_size():
    """the library reads or writes exactly the configured number of elements: the binding
    refuses a state or an output of another size before any call (no GPU needed)"""
    import numpy as np
    from paper_2608_10569_b300 import hweno
    with pytest.raises(ValueError):
        hweno._ptr_of(np.zeros((12, 5, 7)), 12 * 5 * 8)
    with pytest.raises(ValueError):
        hweno._ptr_of(np.zeros((12, 5, 7), dtype=np.float32))
    ptr, dev = hweno._ptr_of(np.zeros((12, 5, 7)), 12 * 5 * 7)
    assert ptr.value and dev == 0
    view = hweno.Solver.__new__(hweno.Solver)
    view.nx, view.ny, view.h, view.lib = 7, 5, None, None
    for call in (lambda: view.set_state(np.zeros((12, 5, 6))),
                 lambda: view.get_state(np.zeros((12, 4, 7))),
                 lambda: view.residual(np.zeros((12, 5, 7)), np.zeros((12, 5, 7))),
                 lambda: view.adjoint_step(np.zeros((12, 5, 7)), 1e-3, np.zeros((12, 5, 8)), np.zeros((12, 5, 7)))):
        with pytest.raises(ValueError):
            call()
    with pytest.raises(ValueError):
        hweno.advance1d([dict(n=8)], [], 0.0, 1.0)


def test_batch_cases_share_the_restart_cap(lib):
    """hweno_batch_step counts restart rounds for all cases together, so the cases of a
    batch must agree on max_halvings"""
    from paper_2608_10569_b300 import hweno
    b = ctypes.c_void_p()
    cfgs = (hweno.hweno_config * 2)(hweno.make_config(8, 8, max_halvings=20), hweno.make_config(8, 8))
    assert lib.hweno_batch_init(cfgs, 2, None, ctypes.byref(b)) == hweno.HWENO_ERR_ARG
    assert b.value is None and b"max_halvings" in lib.hweno_last_error(None)


def test_noalloc_grid_limit_is_checked_before_any_device_call(lib):
    """hweno_residual_noalloc's static scratch holds (ny + 8) * round_up(nx + 8, 16) <= 4096
    padded cells per plane (56 x 56 fills it): 57 x 56 (64 * 80), 56 x 57 (65 * 64),
    400 x 4 (12 * 416) and 4 x 4089 are refused on the host, before any device call,
    with the sizes in the message"""
    from paper_2608_10569_b300 import hweno
    buf = (ctypes.c_double * 12)()
    for nx, ny in ((57, 56), (56, 57), (400, 4), (4, 4089)):
        c = hweno.make_config(nx, ny)
        assert lib.hweno_residual_noalloc(ctypes.byref(c), buf, buf, None, None) == hweno.HWENO_ERR_ARG
        msg = lib.hweno_last_error(None)
        assert b"padded cells" in msg and (b"%d x %d" % (nx, ny)) in msg
