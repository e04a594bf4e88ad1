"""Host logic of the autograd wrapper (autograd.CBESSFM / CBESSFMFunction) on CPU, with a stand-in
plan in place of the library's: which workspace and which taps/ratio state each backward pass
uses, and which forward runs without gradients.  The arithmetic of the real forward and adjoint
is covered by the GPU tests against the oracle; here the stand-in computes y = s x with
s = sum(taps) + ratio, whose gradients are known in closed form."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


class StandInPlan:
    """Same calls as cbessfm.Plan's differentiation form; the "checkpoint" is a copy of x."""

    def __init__(self):
        self.s = None
        self.taps = None
        self.workspaces = 0
        self.plain_calls = 0

    def set_coeffs(self, c):
        self.taps = c.detach().clone()

    def set_ratio(self, r):
        self.s = float(self.taps.sum()) + float(r)

    def new_workspace(self, n_samples, batch=1):
        self.workspaces += 1
        return torch.empty((batch, n_samples, 2), dtype=torch.float64)

    def backpropagate_checkpointed(self, x, ws):
        ws.copy_(x.detach().reshape(ws.shape))
        return x.detach() * self.s

    def backpropagate(self, x):
        self.plain_calls += 1
        return x.detach() * self.s

    def grad(self, gy, ws, want_input=True, want_ratio=True):
        x = ws.reshape(gy.shape)
        dot = float((gy.double() * x).sum())
        gc = torch.full(self.taps.shape, dot, dtype=torch.float64)
        gr = torch.tensor(dot, dtype=torch.float64) if want_ratio else None
        gi = gy * self.s if want_input else None
        return gc, gr, gi


@pytest.fixture(scope="module")
def CBESSFM():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2409_14489_gb300.autograd import CBESSFM
    return CBESSFM


def _module(CBESSFM, taps, ratio):
    return CBESSFM(None, 1, 2, ratio, taps, 16, 4, plan=StandInPlan(), device="cpu")


def test_two_forwards_before_one_backward_use_their_own_checkpoints(CBESSFM):
    """loss = <w1, f(x1)> + <w2, f(x2)>: each backward pass reads its own call's checkpoint, and
    the first call's ratio is reloaded after the second call changed it."""
    rng = np.random.default_rng(1)
    taps = rng.standard_normal((2, 1, 1, 3)).astype(np.float32)
    mod = _module(CBESSFM, taps, 0.25)
    x1, x2, w1, w2 = (torch.from_numpy(rng.standard_normal((10, 2))) for _ in range(4))
    x1.requires_grad_(True)
    x2.requires_grad_(True)
    y1 = mod(x1)
    s1 = float(mod.taps.detach().sum()) + 0.25
    with torch.no_grad():
        mod.ratio.data.fill_(0.75)          # a new state for the second call, without a version bump
    y2 = mod(x2)
    s2 = float(mod.taps.detach().sum()) + 0.75
    ((y1 * w1).sum() + (y2 * w2).sum()).backward()
    dot = float((w1 * x1.detach()).sum() + (w2 * x2.detach()).sum())
    np.testing.assert_allclose(mod.taps.grad.numpy(), np.full(taps.shape, dot), rtol=1e-6)
    assert float(mod.ratio.grad) == pytest.approx(dot, rel=1e-12)
    np.testing.assert_allclose(x1.grad.numpy(), (w1 * s1).numpy(), rtol=1e-6)
    np.testing.assert_allclose(x2.grad.numpy(), (w2 * s2).numpy(), rtol=1e-6)
    assert mod.plan.workspaces == 2


def test_in_place_change_of_the_taps_before_backward_raises(CBESSFM):
    mod = _module(CBESSFM, np.ones((2, 1, 1, 3), np.float32), 0.5)
    y = mod(torch.ones((4, 2), dtype=torch.float64))
    with torch.no_grad():
        mod.taps.mul_(2.0)
    with pytest.raises(RuntimeError, match="inplace"):
        y.sum().backward()


def test_forward_without_gradients_writes_no_checkpoints(CBESSFM):
    mod = _module(CBESSFM, np.ones((2, 1, 1, 3), np.float32), 0.5)
    x = torch.ones((4, 2), dtype=torch.float64)
    with torch.no_grad():
        y = mod(x)
    assert mod.plan.workspaces == 0 and mod.plan.plain_calls == 1
    assert float(y[0, 0]) == pytest.approx(6.5)


def test_ratio_outside_the_unit_interval_is_clamped(CBESSFM):
    mod = _module(CBESSFM, np.zeros((2, 1, 1, 3), np.float32), 0.5)
    with torch.no_grad():
        mod.ratio.fill_(1.7)
    y = mod(torch.ones((4, 2), dtype=torch.float64))
    assert float(mod.ratio.detach()) == 1.0 and float(y.detach()[0, 0]) == pytest.approx(1.0)
