"""Host logic of the gradient helpers, on the CPU: the checkpoint schedule
of gks.checkpointed_gradient, the autograd wrapper gks.make_step_function,
and the wall-force output gks.wall_pressure_force.

The library's State is replaced by a stand-in whose step is a nonlinear
pointwise map and whose adjoint_step is that map's exact transpose at the
given state, so the adjoint chain is right only if every step is applied
once in the primal, every segment is recomputed from its own checkpoint,
and each adjoint step receives the state its forward step started from.
The result is compared with torch.autograd through the same steps run
without checkpoints."""
import numpy as np
import pytest
import torch

from paper_2102_01366_gb300 import gks
from paper_2102_01366_gb300 import inputs as I

NC = 7


def _f(W, dW, dt):
    """one stand-in step: W' = W + dt sin(W) * (1 + |dW|^2 / 15), dW' = dW cos(dt W)"""
    g = 1.0 + (dW * dW).sum(0, keepdim=True) / 15.0
    return W + dt * torch.sin(W) * g, dW * torch.cos(dt * W[:1])


class _FakeState:
    log = []

    torch = torch

    def __init__(self, mesh=None, params=None):
        self.precision = params.precision if params is not None else 0
        self.W = self.dW = None

    def init(self, W, dW):
        self.W, self.dW = W.clone(), dW.clone()

    def step(self, n, dt, t_end):
        for _ in range(n):
            _FakeState.log.append(("step", self.precision))
            # the stand-in's "stage state": a marker of the step's input
            self.stage = (self.W + 100.0, self.dW - 100.0)
            self.W, self.dW = _f(self.W, self.dW, dt)

    def stage_state(self):
        return self.stage[0].clone(), self.stage[1].clone()

    def get(self):
        return self.W.clone(), self.dW.clone()

    def sync(self):
        pass

    def adjoint_step(self, Ws, dWs, lam_W, lam_dW, dt, stage=None):
        _FakeState.log.append(("adjoint", self.precision))
        if stage is not None:
            # the stage state handed over belongs to this very step
            _FakeState.log.append(("staged", self.precision))
            assert torch.equal(stage[0], Ws + 100.0) and torch.equal(stage[1], dWs - 100.0)
        with torch.enable_grad():  # also when called from a backward pass
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


def test_checkpoint_interval_fits_the_memory_budget():
    """Every step where all states fit; otherwise the smallest spacing whose
    checkpoints plus one recomputed segment fit (160 B a cell a state)."""
    assert gks.checkpoint_interval(1000, 200, device="cpu") == 1
    nc, n = 1000, 100
    per = 160 * nc
    frac = 30.0 * per / (1 << 40)  # room for 30 states (a CPU device reports 2^40 B free)
    budget = frac * (1 << 40) / per
    every = gks.checkpoint_interval(nc, n, device="cpu", fraction=frac)
    assert (n // every + every) <= budget < (n // (every - 1) + every - 1)
    assert every > 1


def test_default_spacing_needs_no_recomputation(monkeypatch):
    monkeypatch.setattr(gks, "State", _FakeState)
    _FakeState.log = []
    W0, dW0 = _inputs()
    gks.checkpointed_gradient(_mesh(), gks.params(), W0, dW0, 5, 0.05, _loss, device="cpu")
    # the primal's five steps and five adjoint steps, nothing recomputed; each
    # adjoint step gets its own step's stage state
    assert sum(1 for k, _ in _FakeState.log if k == "step") == 5
    assert sum(1 for k, _ in _FakeState.log if k == "adjoint") == 5
    assert sum(1 for k, _ in _FakeState.log if k == "staged") == 5


def test_fp32_primal_uses_its_own_state_and_fp64_segments(monkeypatch):
    monkeypatch.setattr(gks, "State", _FakeState)
    _FakeState.log = []
    W0, dW0 = _inputs()
    gks.checkpointed_gradient(_mesh(), gks.params(), W0, dW0, 6, 0.05, _loss, checkpoint_every=2,
                              primal_precision=1, device="cpu")
    primal = [p for k, p in _FakeState.log[:6]]
    assert primal == [1] * 6  # the primal run in FP32 bulk
    assert all(p == 0 for _, p in _FakeState.log[6:])  # recomputation and adjoint in FP64


@pytest.mark.parametrize("use_dW", [True, False])
def test_step_function_chain_matches_autograd(use_dW):
    """Four chained applications of make_step_function (backward through
    the state's adjoint step, each step's input kept) against autograd
    through the same steps; with use_dW False the loss ignores the final
    gradients, so the wrapper's backward gets no gradient for them."""
    st = _FakeState()
    dt = 0.09
    step = gks.make_step_function(st, dt)
    W0, dW0 = _inputs()

    def run(fn):
        W = W0.clone().requires_grad_(True)
        dW = dW0.clone().requires_grad_(True)
        Wn, dWn = W, dW
        for _ in range(4):
            Wn, dWn = fn(Wn, dWn)
        J = _loss(Wn) + ((dWn ** 2).sum() if use_dW else 0.0)
        return torch.autograd.grad(J, (W, dW))

    got = run(step)
    ref = run(lambda W, dW: _f(W, dW, dt))
    for a, b in zip(got, ref):
        torch.testing.assert_close(a, b, rtol=1e-13, atol=1e-15)


def test_wall_pressure_force_on_a_closed_wall():
    """The inner sphere of a shell mesh is a closed wall: a uniform pressure
    gives no net force (every wall face found, each with its outward
    sign), and the force's derivative with respect to one wall cell's
    pressure is the sum of A n over that cell's wall faces."""
    mesh = I.sphere_shell_mesh(3, 6, 12, 0.5, 1.5, 1.08)
    g = gks.Mesh(mesh, build_stencils=False)
    force = gks.wall_pressure_force(g, mesh["bkind"], device="cpu")
    gamma = 1.4
    p0 = 0.8
    W = torch.zeros((5, g.nc), dtype=torch.float64)
    W[0] = 1.0
    W[1] = 0.3
    W[4] = p0 / (gamma - 1.0) + 0.5 * 0.3 ** 2
    top, geo = g.topology(), g.geometry()
    kinds = np.asarray(mesh["bkind"]).reshape(g.nc, 4)
    on = (top["nbr"] < 0) & np.isin(kinds, (1, 3))
    area = geo["farea"][top["csr_face"][on]].sum()
    assert 0.9 * np.pi < area < 1.01 * np.pi  # the polyhedral sphere of radius 0.5
    F = force(W)
    assert float(F.abs().max()) < 1e-13 * p0 * area
    # d F / d p of one wall cell, through rho E at fixed rho and rho U
    c = int(np.nonzero(on.any(1))[0][0])
    Wc = W.clone().requires_grad_(True)
    Fx = force(Wc)
    rows = [torch.autograd.grad(Fx[i], Wc, retain_graph=True)[0][4, c] / (gamma - 1.0) for i in range(3)]
    an = np.zeros(3)
    for f in np.nonzero(on[c])[0]:
        e = top["csr_face"][c, f]
        an += geo["farea"][e] * geo["fnorm"][e] * top["csr_sign"][c, f]
    np.testing.assert_allclose([float(r) for r in rows], an, rtol=1e-12, atol=1e-15)
