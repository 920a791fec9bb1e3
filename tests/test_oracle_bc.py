"""Pins of the oracle's inflow and outflow boundaries (Remark 4.1) and of the
rectangular 2D benchmarks built on them (Examples 5.7 and 5.9): the ghost-cell rules as
Remark 4.1 states them, free stream through open faces,
the symmetries of the Sedov and Mach-2000 setups, and the linear-gradient ablation of
Remark 3.1 acting on the gradients alone.
"""
import numpy as np

from oracle import oracle as O
from paper_2608_10569_b300 import inputs as I

G = 4


def test_inflow_and_outflow_ghost_cells():
    """outflow ghosts copy the adjacent interior cell (average and both moments);
    inflow ghosts hold the prescribed state (A inside the band, B outside) with zero
    moments; a y-face inflow fills its whole ghost row, corners included, while an
    x-face inflow column under a y mirror takes the mirror's parity"""
    nx, ny = 10, 8
    case, q = I.random_smooth(nx, ny, seed=12, bc=("symmetry", "symmetry", "symmetry", "symmetry"))
    A = (1.5, 0.6, 0.1, 3.0)
    B = (1.1, 0.2, -0.1, 2.5)
    C = (0.9, 0.0, -0.3, 2.2)
    p = dict(case.params(), bc=("inflow", "outflow", "symmetry", "inflow"),
             inflow=((A, B), None, None, (C, C)), band=((0.5, 0.2), None, None, None))
    g = O.fill_ghosts(O.make_cfg(**p), q)
    dy = 1.0 / ny
    # outflow at x = 1: every ghost column copies column nx - 1 (interior rows)
    for k in range(G):
        assert np.array_equal(g[:, G:G + ny, G + nx + k], g[:, G:G + ny, G + nx - 1])
    # inflow at x = 0: A where the row centre is in the band, B elsewhere; zero moments
    for j in range(ny):
        yc = (j + 0.5) * dy
        st = A if abs(yc - 0.5) < 0.2 else B
        for k in range(G):
            assert np.allclose(g[:4, G + j, k], st, rtol=0, atol=0)
            assert not g[4:, G + j, k].any()
    # inflow at y = 1 fills its ghost rows across the full padded width
    for k in range(G):
        for i in range(nx + 2 * G):
            assert np.array_equal(g[:4, G + ny + k, i], C) and not g[4:, G + ny + k, i].any()
    # symmetry at y = 0 under the x-inflow column: v odd, the eta-moment with the other parity
    for k in range(G):
        row, src = G - 1 - k, G + k
        for i in range(G):
            assert np.array_equal(g[:4, row, i] * np.array([1, 1, -1, 1]), g[:4, src, i])
        # and under the outflow columns: the mirror of the copied interior column
        for i in range(G + nx, nx + 2 * G):
            s = np.array([1, 1, -1, 1])
            assert np.array_equal(g[:4, row, i], s * g[:4, src, i])
            assert np.array_equal(g[8:, row, i], -s * g[8:, src, i])


def test_free_stream_through_inflow_and_outflow():
    """a uniform flow entering through an inflow face with its own state and leaving
    through outflow faces is a steady solution"""
    nx, ny = 12, 10
    U = I.conserved(1.3, 0.7, -0.2, 2.0, 1.4)
    case = I.Case("fs_open", nx, ny, Re=50.0, bc=("inflow", "outflow", "outflow", "inflow"),
                  inflow=((U, U), None, None, (U, U)), band=((0.5, 0.1), None, None, None))
    q = np.zeros((12, ny, nx))
    for v in range(4):
        q[v] = U[v]
    r = O.residual(O.make_cfg(**case.params()), q)
    assert np.abs(r["rhs"]).max() < 1e-13 and np.abs(r["vhat"]).max() < 1e-14


def test_sedov_setup_is_transpose_symmetric():
    """Example 5.7: the corner blast between two reflective faces and two outflow faces
    is its own x <-> y transpose, so the residual is too (to rounding of its scale)"""
    case, q = I.sedov_2d(24)
    r = O.residual(O.make_cfg(**case.params()), q)["rhs"]
    rt = np.zeros_like(r)
    perm = [0, 2, 1, 3]
    for m, m2 in ((0, 0), (1, 2), (2, 1)):
        for v in range(4):
            rt[4 * m2 + perm[v]] = r[4 * m + v].T
    assert np.abs(rt - r).max() <= 1e-13 * np.abs(r).max()
    assert np.abs(r).max() > 0


def test_mach2000_setup_is_mirror_symmetric():
    """Example 5.9: the jet band |y| < 0.05 and the outflow faces are symmetric under
    y -> -y (v and the eta-moment odd), and so is the residual of the initial state"""
    case, q = I.mach2000(32, 16)
    cfg = O.make_cfg(**case.params())
    g = O.fill_ghosts(cfg, q)
    s = np.array([1, 1, -1, 1, 1, 1, -1, 1, -1, -1, 1, -1], dtype=float)[:, None, None]
    assert np.array_equal(g, s * g[:, ::-1, :])
    r = O.residual(cfg, q)["rhs"]
    assert np.abs(r - s * r[:, ::-1, :]).max() <= 1e-13 * np.abs(r).max()
    # the jet enters: the first column's x-momentum grows only inside the band
    yc = -0.25 + (np.arange(16) + 0.5) / 32
    inside = np.abs(yc) < 0.05
    assert (r[1, inside, 0] > 0).all() and np.abs(r[1, ~inside, 0]).max() < 1e-6 * r[1, inside, 0].min()


def test_linear_gradient_ablation_changes_only_the_gradients():
    """Remark 3.1's ablation replaces the nonlinear weights of the gradient
    reconstruction by the linear ones: the traces, volume values, weak moments and
    limiter factors stay, the gradients change"""
    case, q = I.random_rough(20, 18, seed=6, bc=("inflow", "outflow", "symmetry", "outflow"),
                             Re=100.0)
    st = tuple(q[:4, 9, 0])
    p = dict(case.params(), inflow=((st, st), None, None, None), band=((0.5, 0.0), None, None, None))
    a = O.residual(O.make_cfg(**p), q, dumps=True)
    b = O.residual(O.make_cfg(**p, linear_grad=True), q, dumps=True)
    for k in ("face", "vol", "rm", "theta", "vhat"):
        assert np.array_equal(a[k], b[k]), k
    assert np.abs(a["grad"] - b["grad"]).max() > 1e-3 * np.abs(a["grad"]).max()


def test_open_shock_tube_inflow_matches_its_left_state():
    """the open shock tube prescribes its own left state at x = 0: next to that face the
    flow is uniform and at rest, so the residual vanishes there; it lives at the
    diaphragm only"""
    case, q = I.open_shock_tube(32, 16)
    r = O.residual(O.make_cfg(**case.params()), q)["rhs"]
    assert np.abs(r[:, :, :10]).max() <= 1e-12 * np.abs(r).max()
    assert np.abs(r[:, :, 22:]).max() <= 1e-12 * np.abs(r).max()
    assert np.abs(r[:, :, 14:18]).max() > 0
