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
            ref = dWo[3 * q:3 * q + 3]
            scale = np.abs(ref).max()
            if scale > 1e-10:
                assert np.abs(dWg[3 * q:3 * q + 3, c0:c1] - ref).max() / scale < TOL[precision], (k, q)
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
    ms = res["ms_per_step"]
    assert len(ms) == gks.State.NVARIANTS and None not in ms and min(ms) > 0  # precision 1 times all 10
    assert res["fused"] in (0, 1) and s.fused() == res["fused"]
    after = s.get()
    assert cuda.equal(before[0], after[0]) and cuda.equal(before[1], after[1])
    np.testing.assert_array_equal(tb[0], s.case_times()[0])
    # a second state on the same mesh reads the cache
    s2 = gks.State(g, gks.params(weno=1, cfl=0.5, precision=1))
    s2.init(W, dW)
    assert s2.autotune(steps=3, cache=str(tmp_path / "tune.json"))["cached"]


def _rel_state(a, ref):
    """Largest error of each conserved quantity over a case, relative to the
    largest magnitude of that quantity there; the three momentum components
    share one scale (the largest |rho U| entry), so a component that is zero
    at the start (the Riemann slabs' transverse momentum) is not divided by
    its own rounding-level values."""
    mom = np.abs(ref[1:4]).max()
    out = 0.0
    for q in range(5):
        scale = mom if 1 <= q <= 3 else np.abs(ref[q]).max()
        out = max(out, np.abs(a[q] - ref[q]).max() / max(scale, 1e-300))
    return out


def _rel_grad(a, ref):
    """The same for the gradients ([15][n], direction-minor): each
    quantity's three directions share its largest magnitude, the momentum
    components one scale between them; a quantity with no gradient above
    1e-10 is skipped."""
    mom = np.abs(ref[3:12]).max()
    out = 0.0
    for q in range(5):
        scale = mom if 1 <= q <= 3 else np.abs(ref[3 * q:3 * q + 3]).max()
        if scale > 1e-10:
            out = max(out, np.abs(a[3 * q:3 * q + 3] - ref[3 * q:3 * q + 3]).max() / scale)
    return out


def test_batched_workload_full_size_one_step(cuda, oracle_mod):
    """The 48-case batched workload at full size (6,486,324 cells: periodic
    unit cubes of 8^3..40^3 hexes x 6 tets, seed 5, density waves and Riemann
    slabs at Mach 0.5-3), run the way the benchmark times it: FP32 bulk,
    WENO, CFL 0.5, the autotuned variant, one CUDA graph per step.  After one
    step:
      * the two smallest cases (a Riemann slab, 10^3 hexes, and a density
        wave, 12^3) match the oracle element by element, averages and
        gradients, at the FP32 tolerance;
      * every case conserves mass, momentum and energy to FP64 rounding
        (each face record enters its two cells with opposite signs, and the
        cell sums are FP64);
      * every case's cell averages agree with the FP64 path within the FP32
        tolerance, and the FP64 path matches the oracle on the sampled cases
        at 1e-11;
      * every case's gradients agree with the FP64 path within the FP32
        tolerance.  (The gradients are evolved from the face states by the
        divergence theorem, Sec. 3, Eq. step-du; the FP32 path takes the
        face states relative to the mean of the two cell averages, so their
        rounding is not multiplied by the 3 / dr of the cells.)"""
    batch, W, dW, desc, meshes = I.batch_cases(n_cases=48, n_range=(8, 40), seed=5)
    g = gks.Mesh(batch)
    first = g.case_first
    assert g.ncase == 48 and g.nc == 6486324
    geo = g.geometry()
    vol, dr = geo["vol"], geo["dr"]
    res = {}
    for precision in (1, 0):
        s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=precision))
        s.init(W, dW)
        if precision == 1:
            s.autotune(steps=5, cache=False)  # restores the initial state
        s.step(1)
        s.sync()
        res[precision] = [x.cpu().numpy() for x in s.get()] + [s.case_times()[0]]
        del s
        cuda.cuda.empty_cache()

    # sampled cases against the oracle, both precisions
    sample = sorted(range(48), key=lambda k: desc[k]["n"])[:2]
    assert {desc[k]["kind"] for k in sample} == {"sine", "riemann"}
    p = oracle_mod.params(weno=1, cfl=0.5)
    for k in sample:
        c0, c1 = first[k], first[k + 1]
        Wo, dWo, to, _ = oracle_mod.Mesh(meshes[k]).run(p, W[:, c0:c1], dW[:, c0:c1], nsteps=1)
        for precision, (Wg, dWg, tg) in res.items():
            assert abs(tg[k] - to) <= TOL[precision] * to, (k, precision)
            assert _rel_state(Wg[:, c0:c1], Wo) < TOL[precision], (k, precision)
            assert _rel_grad(dWg[:, c0:c1], dWo) < TOL[precision], (k, precision)

    # every case: conservation and FP32 against FP64
    W32, dW32, t32 = res[1]
    W64, dW64, t64 = res[0]
    # the FP32 path forms its time step from its FP32 copy of the state
    np.testing.assert_allclose(t32, t64, rtol=TOL[1], atol=0)
    worst = {"drift": 0.0, "state": 0.0, "grad": 0.0}
    for k in range(48):
        c0, c1 = first[k], first[k + 1]
        v = vol[c0:c1]
        total0 = W[:, c0:c1] @ v
        scale = (np.abs(W[:, c0:c1]) @ v).max()
        for Wg in (W32, W64):
            drift = np.abs(Wg[:, c0:c1] @ v - total0).max()
            assert drift <= 1e-11 * scale, (k, drift / scale)
            worst["drift"] = max(worst["drift"], drift / scale)
        state = _rel_state(W32[:, c0:c1], W64[:, c0:c1])
        assert state < TOL[1], (k, state)
        worst["state"] = max(worst["state"], state)
        grad = _rel_grad(dW32[:, c0:c1], dW64[:, c0:c1])
        assert grad < TOL[1], (k, desc[k], grad)
        worst["grad"] = max(worst["grad"], grad)
    print("batched full size, worst over 48 cases:", {k: float("%.3g" % v) for k, v in worst.items()})


def _orderings_case(kind):
    if kind == "batch":
        batch, W, dW, desc, meshes = I.batch_cases(n_cases=3, n_range=(3, 5), seed=13)
        return batch, W, dW, dict(weno=1, cfl=0.5)
    if kind == "sod":
        mesh, W, dW = I.sod_case(nx=16, nyz=3)
        return mesh, W, dW, dict(weno=1, cfl=0.5)
    # the sphere shell: non-slip wall, far field held fixed, viscous, Pr fix
    mesh = I.sphere_shell_mesh(3, 6, 12, 0.5, 1.5, 1.08)
    W, dW = I.sine_wave_state(mesh, amp=0.2, k=2.0, u=(0.35, 0.15, 0.0), p=1 / 1.4)
    return mesh, W, dW, dict(weno=1, cfl=0.5, viscous=1, mu=0.01, prandtl=0.72)


@pytest.mark.parametrize("kind", ["batch", "sod", "shell"])
@pytest.mark.parametrize("precision", [1, 2])
def test_cell_orderings_give_bit_identical_results(cuda, kind, precision):
    """The device cell orderings (caller's, reverse Cuthill-McKee, Morton)
    change memory locality only: every cell and face computes the same
    arithmetic in the same order, so states, gradients, case times and the
    reconstruction diagnostics are bit-identical, with either face order
    and the separate slopes pass; and re-ordering mid-run carries the state
    over exactly."""
    mesh, W, dW, kw = _orderings_case(kind)
    g = gks.Mesh(mesh)
    ref = None
    for order in (0, 1, 2):
        for variant in ((0, 3, 0), (1, 3, 1)):
            s = gks.State(g, gks.params(precision=precision, **kw))
            s.set_cell_order(order)
            s.set_variant(*variant)
            s.init(W, dW)
            s.step(3)
            s.sync()
            out = [x.cpu() for x in s.get()] + [cuda.tensor(s.case_times()[0])] + \
                  [x.cpu() for x in s.debug_reconstruct()]
            if ref is None:
                ref = out
            else:
                for a, b in zip(ref, out):
                    assert cuda.equal(a, b), (order, variant)
    # re-order between steps: 3 steps, Morton, 3 steps, RCM, 2 steps, caller's
    s = gks.State(g, gks.params(precision=precision, **kw))
    s.init(W, dW)
    s.step(3)
    s.set_cell_order(2)
    s.step(3)
    s.set_cell_order(1)
    s.step(2)
    s.set_cell_order(0)
    s.sync()
    a = [x.cpu() for x in s.get()]
    s2 = gks.State(g, gks.params(precision=precision, **kw))
    s2.init(W, dW)
    s2.step(8)
    s2.sync()
    b = [x.cpu() for x in s2.get()]
    for x, y in zip(a, b):
        assert cuda.equal(x, y)


def test_autotune_over_orderings_restores_state(cuda):
    batch, W, dW, desc, meshes = I.batch_cases(n_cases=3, n_range=(3, 5), seed=11)
    g = gks.Mesh(batch)
    s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=1))
    s.init(W, dW)
    s.step(2)
    s.sync()
    before = [x.clone() for x in s.get()]
    res = s.autotune(steps=2, cache=False, orders=True)
    assert res["cell_order"] in (0, 1, 2) and len(res["ms_per_order"]) == 3
    after = s.get()
    assert cuda.equal(before[0], after[0]) and cuda.equal(before[1], after[1])
    # FP64 states keep the caller's order
    s64 = gks.State(g, gks.params(weno=1, cfl=0.5, precision=0))
    with pytest.raises(gks.GksError) as e:
        s64.set_cell_order(1)
    assert e.value.status == -8
