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


@pytest.mark.parametrize("precision", [0, 1])
def test_variants_give_identical_results(cuda, precision):
    """Execution variants change speed only.  The face order leaves every
    face's arithmetic unchanged: bit-identical state.  The two FP32 flux
    occupancy variants are separately optimised instantiations of the same
    code (the compiler may contract differently), and so are the fused and
    the separate slopes passes: equal to the working precision's tolerance."""
    mesh, W, dW = I.sod_case(nx=16, nyz=3)
    g = gks.Mesh(mesh)
    res = {}
    for v in ((0, 3, 0), (1, 3, 0), (0, 2, 0), (1, 2, 0), (0, 3, 1), (1, 2, 1)):
        s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=precision))
        s.set_variant(*v)
        s.init(W, dW)
        s.step(3)
        s.sync()
        res[v] = [x.cpu() for x in s.get()] + [s.debug_face_records(1e-3, 1).cpu()]
    for fb in (3, 2):
        for a, b in zip(res[(0, fb, 0)], res[(1, fb, 0)]):
            assert cuda.equal(a, b)
    tol = 1e-13 if precision == 0 else 2e-5
    for other in ((0, 2, 0), (0, 3, 1), (1, 2, 1)):
        for a, b in zip(res[(0, 3, 0)], res[other]):
            if precision == 0 and other[2] == 0:
                assert cuda.equal(a, b)
            else:
                assert float((a - b).abs().max() / b.abs().max()) < tol, other


def test_set_variant_rejects_bad_values(cuda):
    mesh, W, dW = I.sod_case(nx=8, nyz=2)
    s = gks.State(gks.Mesh(mesh), gks.params(weno=1))
    for bad in ((2, 3, 0), (0, 4, 0), (0, 3, 2)):
        st = gks.lib().gks_state_set_variant(s._h, *bad)
        assert st == -1, bad  # GKS_E_ARG


def test_autotune_restores_state(cuda, tmp_path):
    batch, W, dW, desc, meshes = I.batch_cases(n_cases=3, n_range=(3, 5), seed=11)
    g = gks.Mesh(batch)
    s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=1))
    s.init(W, dW)
    s.step(2)
    s.sync()
    before = [x.clone() for x in s.get()]
    tb = s.case_times()
    res = s.autotune(steps=3, cache=str(tmp_path / "tune.json"))
    fo, fb, sp = res["variant"]
    assert fo in (0, 1) and fb in (2, 3) and sp in (0, 1) and not res["cached"]
    assert len(res["ms_per_step"]) == 8 and min(res["ms_per_step"]) > 0
    after = s.get()
    assert cuda.equal(before[0], after[0]) and cuda.equal(before[1], after[1])
    np.testing.assert_array_equal(tb[0], s.case_times()[0])
    # a second state on the same mesh reads the cache
    s2 = gks.State(g, gks.params(weno=1, cfl=0.5, precision=1))
    s2.init(W, dW)
    assert s2.autotune(steps=3, cache=str(tmp_path / "tune.json"))["cached"]
