"""The host logic of hweno.rollout's autograd function, with a stand-in for the solver
(no device): which adjoint calls the backward makes, in which order, and what it does
when the forward's request for kept intermediates was refused for lack of memory."""
import pytest

torch = pytest.importorskip("torch")

from paper_2608_10569_b300 import hweno  # noqa: E402


class FakeSolver:
    """records the calls of the rollout; reserve grants intermediates or not"""
    log = []
    grant = True

    def __init__(self, params, precision="fp64"):
        self.q = None
        self.closed = False
        FakeSolver.log.append(("init",))

    def set_state(self, q):
        self.q = q.clone()

    def get_state(self):
        return self.q

    def step(self):
        self.q = self.q * 1.0
        return 1e-3, 0

    def adjoint_init(self):
        FakeSolver.log.append(("adjoint_init",))

    def adjoint_reserve(self, n, keep_intermediates=True):
        FakeSolver.log.append(("reserve", n))
        return FakeSolver.grant and keep_intermediates

    def adjoint_record(self, on):
        FakeSolver.log.append(("record", on))

    def adjoint_replay(self, lam):
        FakeSolver.log.append(("replay",))
        return lam, 0.5

    def adjoint_segment(self, q, dts, lam):
        FakeSolver.log.append(("segment", len(dts)))
        return lam, 0.25

    def close(self):
        self.closed = True
        FakeSolver.log.append(("close",))


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(hweno, "Solver", FakeSolver)
    if "_ROLLOUT" in vars(hweno):
        monkeypatch.delattr(hweno, "_ROLLOUT")
    FakeSolver.log = []
    yield FakeSolver


@pytest.mark.parametrize("grant", [True, False])
def test_backward_replays_the_recording_without_reserving_again(fake, grant):
    """the forward reserved and recorded the final segment; the backward replays it and
    recomputes the earlier segments in the same storage, whether or not the forward's
    intermediates were granted: no second reservation, which could drop the recording"""
    fake.grant = grant
    q0 = torch.ones(12, 4, 4, dtype=torch.float64, requires_grad=True)
    mu = torch.tensor(1e-3, dtype=torch.float64, requires_grad=True)
    qT = hweno.rollout(q0, mu, {"nx": 4, "ny": 4}, nsteps=7, ckpt=3)
    qT.sum().backward()
    calls = [c[0] for c in fake.log]
    assert calls.count("reserve") == 1 and calls.index("reserve") < calls.index("record")
    assert ("replay",) in fake.log and fake.log.count(("segment", 3)) == 2
    assert calls[-1] == "close"
    assert float(mu.grad) == pytest.approx(0.5 + 2 * 0.25)


def test_second_backward_is_refused(fake):
    q0 = torch.ones(12, 4, 4, dtype=torch.float64, requires_grad=True)
    qT = hweno.rollout(q0, 1e-3, {"nx": 4, "ny": 4}, nsteps=2, ckpt=2)
    y = qT.sum()
    y.backward(retain_graph=True)
    with pytest.raises(RuntimeError):
        y.backward()


def test_forward_without_gradient_releases_the_solver(fake):
    q0 = torch.ones(12, 4, 4, dtype=torch.float64)
    with torch.no_grad():
        hweno.rollout(q0, 1e-3, {"nx": 4, "ny": 4}, nsteps=3, ckpt=2)
    assert ("close",) in fake.log and ("reserve", 2) not in fake.log
