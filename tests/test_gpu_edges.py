"""Degenerate inputs on the GPU path, against the oracle.

A single hexahedron split into 6 tetrahedra: every cell has only 2
neighbours, so every reconstruction stencil is singular and every cell
falls back to its average (first order, Sec. 4.4's "fewer than 3 neighbours"
case); every cell also has 2 boundary faces.  With open ends, and closed by
slip walls on all six sides (mass and energy then conserved), the GPU path
must follow the oracle step by step in both precisions.  Block and warp
raggedness (cell counts that are not multiples of 24, face counts that are
not multiples of 32) is covered by the parity cases of test_gpu_parity."""
import numpy as np
import pytest

from paper_2102_01366_gb300 import gks
from paper_2102_01366_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {0: 1e-11, 1: 2e-5}


@pytest.fixture(scope="module")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")
    from paper_2102_01366_gb300 import _build
    _build.build()
    gks.lib()
    return torch


def _single_hex(walls):
    mesh = I.box_mesh((1, 1, 1), (1.0, 1.0, 1.0), (False, False, False), jitter=0.0, seed=0)
    if walls:
        mesh["bkind"] = I.wall_kinds(mesh, (0, 1, 2))
    return mesh


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("precision", [0, 1])
def test_single_hexahedron(cuda, oracle_mod, precision, walls):
    mesh = _single_hex(walls)
    W, dW = I.riemann_x_state(mesh, left=(1.0, 0.2, 1.0), right=(0.5, 0.2, 0.6), x0=0.45)
    g = gks.Mesh(mesh)
    assert g.n_singular == 6
    o = oracle_mod.Mesh(mesh)
    p = oracle_mod.params(weno=1, cfl=0.5)
    Wo, dWo, t_o, _ = o.run(p, W, dW, nsteps=5)
    s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=precision))
    s.init(W, dW)
    s.step(5)
    s.sync()
    Wg, dWg = [x.cpu().numpy() for x in s.get()]
    for q in range(5):
        scale = max(np.abs(Wo[q]).max(), 1e-300)
        assert np.abs(Wg[q] - Wo[q]).max() / scale < TOL[precision], q
    gscale = max(np.abs(dWo).max(), 1e-300)
    assert np.abs(dWg - dWo).max() / gscale < TOL[precision]
    if walls:
        vol = g.geometry()["vol"]
        for q in (0, 4):
            assert abs((Wg[q] * vol).sum() - (W[q] * vol).sum()) < 10 * TOL[precision] * abs((W[q] * vol).sum())


def test_bounded_wait_gives_up_with_a_status_and_the_state_stays_usable(cuda, oracle_mod):
    """The failure path of the bounded device waits, without a GPU fault:
    the reconstruction's mbarrier wait, run on a barrier that nothing
    completes (no copy in flight), gives up after its polls, the device
    error flag reaches the host as GKS_E_TIMEOUT with its message, and the
    same state then steps normally (matching the oracle)."""
    mesh, W, dW = I.sine_wave_case(n=3)
    g = gks.Mesh(mesh)
    s = gks.State(g, gks.params(weno=1, cfl=0.5))
    s.init(W, dW)
    for tries in (0, 8):
        assert s.debug_wait_timeout(tries) == -6  # GKS_E_TIMEOUT
        assert b"bounded device wait" in gks.lib().gks_last_error()
    s.init(W, dW)
    s.step(1)
    s.sync()
    Wg = s.get()[0].cpu().numpy()
    Wo, _, _, _ = oracle_mod.Mesh(mesh).run(oracle_mod.params(weno=1, cfl=0.5), W, dW, nsteps=1)
    assert max(np.abs(Wg[q] - Wo[q]).max() / np.abs(Wo[q]).max() for q in range(5)) < 1e-11
