"""The checkpoint schedule of gks.checkpointed_gradient (host logic, no GPU).

The library's State is replaced by a stand-in whose step is a nonlinear
pointwise map and whose adjoint_step is that map's exact transpose at the
given state, so the adjoint chain is right only if every step is applied
once in the primal, every segment is recomputed from its own checkpoint,
and each adjoint step receives the state its forward step started from.
The result is compared with torch.autograd through the same steps run
without checkpoints."""
import pytest
import torch

from paper_2102_01366_gb300 import gks

NC = 7


def _f(W, dW, dt):
    """one stand-in step: W' = W + dt sin(W) * (1 + |dW|^2 / 15), dW' = dW cos(dt W)"""
    g = 1.0 + (dW * dW).sum(0, keepdim=True) / 15.0
    return W + dt * torch.sin(W) * g, dW * torch.cos(dt * W[:1])


class _FakeState:
    log = []

    def __init__(self, mesh, params):
        self.precision = params.precision
        self.W = self.dW = None

    def init(self, W, dW):
        self.W, self.dW = W.clone(), dW.clone()

    def step(self, n, dt, t_end):
        for _ in range(n):
            _FakeState.log.append(("step", self.precision))
            self.W, self.dW = _f(self.W, self.dW, dt)

    def get(self):
        return self.W.clone(), self.dW.clone()

    def sync(self):
        pass

    def adjoint_step(self, Ws, dWs, lam_W, lam_dW, dt):
        _FakeState.log.append(("adjoint", self.precision))
        W = Ws.clone().requires_grad_(True)
        dW = dWs.clone().requires_grad_(True)
        W1, dW1 = _f(W, dW, dt)
        gW, gdW = torch.autograd.grad((W1, dW1), (W, dW), (lam_W, lam_dW))
        return gW, gdW


def _mesh():
    m = gks.Mesh.__new__(gks.Mesh)  # no library handle
    m._h = None
    m.nc = NC
    return m


def _loss(W):
    return (W[1:4] ** 2 / W[:1]).sum() / 2.0


def _inputs():
    g = torch.Generator().manual_seed(3)
    W = 1.0 + 0.5 * torch.rand((5, NC), generator=g, dtype=torch.float64)
    dW = torch.rand((15, NC), generator=g, dtype=torch.float64) - 0.5
    return W, dW


@pytest.mark.parametrize("nsteps,every", [(7, 3), (6, 3), (5, 1), (4, 10), (1, 1), (9, 2)])
def test_checkpointed_gradient_matches_autograd(monkeypatch, nsteps, every):
    monkeypatch.setattr(gks, "State", _FakeState)
    _FakeState.log = []
    W0, dW0 = _inputs()
    dt = 0.07
    J, gW, gdW = gks.checkpointed_gradient(_mesh(), gks.params(), W0, dW0, nsteps, dt, _loss,
                                           checkpoint_every=every, device="cpu")
    W = W0.clone().requires_grad_(True)
    dW = dW0.clone().requires_grad_(True)
    Wn, dWn = W, dW
    for _ in range(nsteps):
        Wn, dWn = _f(Wn, dWn, dt)
    Jr = _loss(Wn)
    rW, rdW = torch.autograd.grad(Jr, (W, dW))
    jr = float(Jr.detach())
    assert abs(J - jr) <= 1e-14 * abs(jr)
    torch.testing.assert_close(gW, rW, rtol=1e-13, atol=1e-15)
    torch.testing.assert_close(gdW, rdW, rtol=1e-13, atol=1e-15)
    # work: the primal once, each segment recomputed minus its first step,
    # one adjoint step per forward step
    nseg = len([n for n in range(0, nsteps, every)])
    steps = sum(1 for k, _ in _FakeState.log if k == "step")
    assert steps == nsteps + (nsteps - nseg)
    assert sum(1 for k, _ in _FakeState.log if k == "adjoint") == nsteps


def test_fp32_primal_uses_its_own_state_and_fp64_segments(monkeypatch):
    monkeypatch.setattr(gks, "State", _FakeState)
    _FakeState.log = []
    W0, dW0 = _inputs()
    gks.checkpointed_gradient(_mesh(), gks.params(), W0, dW0, 6, 0.05, _loss, checkpoint_every=2,
                              primal_precision=1, device="cpu")
    primal = [p for k, p in _FakeState.log[:6]]
    assert primal == [1] * 6  # the primal run in FP32 bulk
    assert all(p == 0 for _, p in _FakeState.log[6:])  # recomputation and adjoint in FP64
