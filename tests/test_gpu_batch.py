"""Batched cases (one mesh of disjoint components, per-case time step)
against the oracle run case by case."""
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


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_cases_run_alone(cuda, oracle_mod, precision):
    batch, W, dW, desc, meshes = I.batch_cases(n_cases=4, n_range=(2, 4), seed=3)
    g = gks.Mesh(batch)
    s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=precision))
    s.init(W, dW)
    s.step(5)
    s.sync()
    Wg, dWg = [x.cpu().numpy() for x in s.get()]
    tg, dtg = s.case_times()
    p = oracle_mod.params(weno=1, cfl=0.5)
    for k, m in enumerate(meshes):
        c0, c1 = g.case_first[k], g.case_first[k + 1]
        om = oracle_mod.Mesh(m)
        Wo, dWo, to, _ = om.run(p, W[:, c0:c1], dW[:, c0:c1], nsteps=5)
        assert abs(tg[k] - to) <= TOL[precision] * to
        for q in range(5):
            ref = Wo[q]
            scale = max(np.abs(ref).max(), 1e-300)
            assert np.abs(Wg[q, c0:c1] - ref).max() / scale < TOL[precision], (k, q)
    # the cases did get different steps
    assert len(set(np.round(dtg, 12))) > 1


def test_batch_t_end_per_case(cuda):
    batch, W, dW, desc, meshes = I.batch_cases(n_cases=3, n_range=(2, 4), seed=7)
    g = gks.Mesh(batch)
    s = gks.State(g, gks.params(weno=1, cfl=0.5))
    s.init(W, dW)
    t_end = 0.05
    s.run(t_end=t_end, chunk=8)
    t, dt = s.case_times()
    np.testing.assert_allclose(t, t_end, rtol=0, atol=1e-14)
    Wa, _ = s.get()
    s.step(2, 0.0, t_end)
    s.sync()
    Wb, _ = s.get()
    assert cuda.equal(Wa, Wb)
