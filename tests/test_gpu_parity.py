"""GPU path (through the C ABI) against the FP64 CPU oracle, element by
element on the same seeded inputs.

Tolerances (normwise relative per component, max|gpu - oracle| / max|oracle|):
FP64 path 1e-11 after 10 steps; FP32-bulk path 2e-5.  Connectivity is
compared bit for bit on the host (test_abi_host)."""
import math

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


def _rel(a, b, axis=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.abs(b).max(axis=axis, keepdims=axis is not None)
    scale = np.maximum(scale, 1e-300)
    return (np.abs(a - b).max(axis=axis, keepdims=axis is not None) / scale).max()


def _state_rel(Wg, Wo):
    """max over components of the normwise relative error (rows = components)."""
    return max(_rel(Wg[q], Wo[q]) for q in range(Wo.shape[0]))


CASES = {
    # name: (mesh factory, state factory, oracle params kwargs)
    "sine_n3_linear": (lambda: I.box_mesh((3, 3, 3), jitter=0.1, seed=31, diagonal=(1, 1, -1)),
                       lambda m: I.sine_wave_state(m), dict(weno=0)),
    "sine_n3_weno": (lambda: I.box_mesh((3, 3, 3), jitter=0.1, seed=32),
                     lambda m: I.sine_wave_state(m), dict(weno=1)),
    "sine_n2_weno2": (lambda: I.box_mesh((2, 2, 2), jitter=0.1, seed=33),
                      lambda m: I.sine_wave_state(m), dict(weno=1, order=2)),
    "sod_small_weno": (lambda: I.box_mesh((12, 2, 2), (1.0, 1 / 6, 1 / 6), (False, True, True), jitter=0.1,
                                          seed=34),
                       lambda m: I.riemann_x_state(m), dict(weno=1)),
    "sine_n3_smooth_viscous": (lambda: I.box_mesh((3, 3, 3), jitter=0.1, seed=35),
                               lambda m: I.sine_wave_state(m), dict(weno=1, smooth_flux=1, viscous=1, mu=1e-3)),
    # the Pr fix (Pr = 0.72) on the full and the smooth viscous solver
    "sine_n3_viscous_prandtl": (lambda: I.box_mesh((3, 3, 3), jitter=0.1, seed=36),
                                lambda m: I.sine_wave_state(m), dict(weno=1, viscous=1, mu=1e-2, prandtl=0.72)),
    "sine_n3_smooth_viscous_prandtl": (lambda: I.box_mesh((3, 3, 3), jitter=0.1, seed=39),
                                       lambda m: I.sine_wave_state(m),
                                       dict(weno=0, smooth_flux=1, viscous=1, mu=1e-2, prandtl=0.72)),
    # slip walls at both x ends (Sec. 4.4), y and z periodic
    "closed_box_weno": (lambda: _walled(I.box_mesh((4, 2, 2), (1.0, 0.5, 0.5), (False, True, True), jitter=0.1,
                                                   seed=36)),
                        lambda m: I.sine_wave_state(m, k=4.0 * math.pi, u=(0.6, -0.3, 0.2)), dict(weno=1)),
    "closed_box_linear_order2": (lambda: _walled(I.box_mesh((4, 2, 2), (1.0, 0.5, 0.5), (False, True, True),
                                                            jitter=0.1, seed=37)),
                                 lambda m: I.sine_wave_state(m, k=4.0 * math.pi, u=(-0.5, 0.2, 0.1)),
                                 dict(weno=1, order=2)),
    "wall_reflection_weno": (lambda: I.wall_reflection_case(nx=8, nyz=2)[0],
                             lambda m: I.riemann_x_state(m, left=(1.0, 1.0, 1.0), right=(1.0, 1.0, 1.0)),
                             dict(weno=1)),
    # non-slip adiabatic walls, viscous solver
    "noslip_box_viscous": (lambda: _noslip(I.box_mesh((4, 2, 2), (1.0, 0.5, 0.5), (False, True, True), jitter=0.1,
                                                      seed=38)),
                           lambda m: I.sine_wave_state(m, k=4.0 * math.pi, u=(0.6, -0.3, 0.2)),
                           dict(weno=1, viscous=1, mu=0.01)),
    # non-slip isothermal walls (Sec. 4.4) at T_w = 0.9, viscous
    "isothermal_box_viscous": (lambda: _isothermal(I.box_mesh((4, 2, 2), (1.0, 0.5, 0.5), (False, True, True),
                                                              jitter=0.1, seed=42)),
                               lambda m: I.sine_wave_state(m, k=4.0 * math.pi, u=(0.3, -0.2, 0.1)),
                               dict(weno=1, viscous=1, mu=0.01, wall_temperature=0.9)),
    # a non-slip wall at x = 0 and a wall moving along y and z at x = 1, viscous
    "moving_wall_box_viscous": (lambda: _moving(I.box_mesh((4, 2, 2), (1.0, 0.5, 0.5), (False, True, True),
                                                           jitter=0.1, seed=45)),
                                lambda m: I.sine_wave_state(m, k=4.0 * math.pi, u=(0.3, -0.2, 0.1)),
                                dict(weno=1, viscous=1, mu=0.01, wall_velocity=(0.0, 0.4, -0.2))),
    # the sphere's O-type shell (pole rows of 3 tets per hexahedron), non-slip
    # wall at r = 0.5, far field held at r = 1.5, viscous, a perturbed free
    # stream; with linear weights the wall cells take the first-order fit
    "sphere_shell_linear_viscous": (lambda: I.sphere_shell_mesh(3, 6, 12, 0.5, 1.5, 1.08),
                                    lambda m: I.sine_wave_state(m, amp=0.2, k=2.0, u=(0.35, 0.15, 0.0), p=1 / 1.4),
                                    dict(weno=0, viscous=1, mu=0.01, prandtl=0.72)),
    "sphere_shell_weno_viscous": (lambda: I.sphere_shell_mesh(3, 6, 12, 0.5, 1.5, 1.08),
                                  lambda m: I.sine_wave_state(m, amp=0.2, k=2.0, u=(0.35, 0.15, 0.0), p=1 / 1.4),
                                  dict(weno=1, viscous=1, mu=0.01, prandtl=0.72)),
    # Sec. 4.4 constrained least squares for the momenta of the non-slip wall
    # cells (wall velocity zero at the wall face centroids in step 1, at the
    # wall Gauss points in step 2): WENO, linear weights, second order
    "noslip_box_constrained_weno": (lambda: _noslip(I.box_mesh((4, 2, 2), (1.0, 0.5, 0.5), (False, True, True),
                                                               jitter=0.1, seed=46)),
                                    lambda m: I.sine_wave_state(m, k=4.0 * math.pi, u=(0.6, -0.3, 0.2)),
                                    dict(weno=1, viscous=1, mu=0.01, wall_constraint=1)),
    "noslip_box_constrained_linear": (lambda: _noslip(I.box_mesh((4, 2, 2), (1.0, 0.5, 0.5), (False, True, True),
                                                                 jitter=0.1, seed=47)),
                                      lambda m: I.sine_wave_state(m, k=4.0 * math.pi, u=(0.3, 0.4, -0.2)),
                                      dict(weno=0, viscous=1, mu=0.01, wall_constraint=1)),
    "noslip_box_constrained_order2": (lambda: _noslip(I.box_mesh((4, 2, 2), (1.0, 0.5, 0.5), (False, True, True),
                                                                 jitter=0.1, seed=48)),
                                      lambda m: I.sine_wave_state(m, k=4.0 * math.pi, u=(-0.4, 0.2, 0.3)),
                                      dict(weno=1, order=2, viscous=1, mu=0.01, wall_constraint=1)),
    "sphere_shell_constrained_weno": (lambda: I.sphere_shell_mesh(3, 6, 12, 0.5, 1.5, 1.08),
                                      lambda m: I.sine_wave_state(m, amp=0.2, k=2.0, u=(0.35, 0.15, 0.0),
                                                                  p=1 / 1.4),
                                      dict(weno=1, viscous=1, mu=0.01, prandtl=0.72, wall_constraint=1)),
    # both ends fixed to the initial state (inflow state, wave profile)
    "shu_osher_small_weno": (lambda: I.shu_osher_case(nx=20, nyz=2, jitter=0.1)[0],
                             lambda m: I.shu_osher_state(m), dict(weno=1)),
}


# Cases whose step amplifies rounding: on the coarse shell (22.5 degrees
# between neighbouring wall faces) the third-order WENO wall cells grow a
# 1e-15 relative perturbation of the start to 3e-13 after 5 steps and 1e-10
# after 10 in the oracle itself (the same run twice, once perturbed; with
# linear weights it stays at 8e-15), so two implementations can agree to the
# stated tolerance only over the first steps; those cases compare fewer.
STEPS = {"sphere_shell_weno_viscous": 4, "sphere_shell_constrained_weno": 4}


def _walled(mesh):
    mesh["bkind"] = I.wall_kinds(mesh, (0,))
    return mesh


def _moving(mesh):
    mesh["bkind"] = I.boundary_kinds(mesh, {(0, "lo"): I.BC_NOSLIP_WALL, (0, "hi"): I.BC_MOVING_WALL})
    return mesh


def _isothermal(mesh):
    mesh["bkind"] = I.boundary_kinds(mesh, {(0, "lo"): I.BC_ISOTHERMAL_WALL, (0, "hi"): I.BC_ISOTHERMAL_WALL})
    return mesh


def _noslip(mesh):
    mesh["bkind"] = I.boundary_kinds(mesh, {(0, "lo"): I.BC_NOSLIP_WALL, (0, "hi"): I.BC_NOSLIP_WALL})
    return mesh


def _setup(cuda, oracle_mod, name, precision):
    mk, st, kw = CASES[name]
    mesh = mk()
    W, dW = st(mesh)
    # fixed boundary faces hold the initial state (as gks_init_state does)
    mesh["fixed_state"] = (W, dW)
    kw = dict(kw)
    kw.setdefault("cfl", 0.5)
    g = gks.Mesh(mesh)
    s = gks.State(g, gks.params(precision=precision, **kw))
    s.init(W, dW)
    o = oracle_mod.Mesh(mesh)
    return mesh, W, dW, s, o, oracle_mod.params(**kw)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", sorted(CASES))
def test_reconstruction_parity(cuda, oracle_mod, name, precision):
    """Both paths against the oracle on the same FP64 state.  The FP32 path
    keeps each cell average as an FP32 hi / lo pair, so the differences
    between neighbouring averages (which can be far smaller than the
    averages, e.g. the energy of a slow flow) are exact to their own FP32
    rounding."""
    mesh, W, dW, s, o, p = _setup(cuda, oracle_mod, name, precision)
    poly_g, slopes_g, fb_g = [x.cpu().numpy() for x in s.debug_reconstruct()]
    poly_o, slopes_o, fb_o = o.reconstruct(p, W, dW)
    np.testing.assert_array_equal(fb_g, fb_o)
    tol = TOL[precision]
    for q in range(5):
        # each coefficient family relative to its own size
        for lo, hi in ((0, 1), (1, 4), (4, 10)):
            if np.abs(poly_o[:, q, lo:hi]).max() > 1e-12:
                assert _rel(poly_g[:, q, lo:hi], poly_o[:, q, lo:hi]) < tol, (q, lo)
    if p.weno or p.order == 2:
        assert _rel(slopes_g, slopes_o) < tol


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("stage", [1, 2])
@pytest.mark.parametrize("name", sorted(CASES))
def test_face_record_parity(cuda, oracle_mod, name, stage, precision):
    mesh, W, dW, s, o, p = _setup(cuda, oracle_mod, name, precision)
    dt = o.timestep(p, W)
    rec_g = s.debug_face_records(dt, stage).cpu().numpy()
    rec_o = o.face_records(p, W, dW, dt, stage)
    # column groups: flux parts (5 each) and gradient parts (15 each)
    groups = [(0, 5), (5, 10), (10, 25), (25, 40)] if stage == 1 else [(0, 5), (5, 20)]
    # a group that vanishes analytically (W(dt) - W(0) of a uniform state)
    # is compared against 1e-3 w |W|, far above either precision's noise
    floor = 1e-3 * o.geometry()["farea"].max() / 3.0 * np.abs(W).max()
    for lo, hi in groups:
        ref = rec_o[:, lo:hi]
        scale = max(np.abs(ref).max(), floor)
        err = np.abs(rec_g[:, lo:hi] - ref).max() / scale
        assert err < TOL[precision], (lo, hi, err)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", sorted(CASES))
def test_ten_steps_parity(cuda, oracle_mod, name, precision):
    mesh, W, dW, s, o, p = _setup(cuda, oracle_mod, name, precision)
    nsteps = STEPS.get(name, 10)
    Wo, dWo, t_o, n = o.run(p, W, dW, nsteps=nsteps)
    s.step(nsteps)
    s.sync()
    Wg, dWg = [x.cpu().numpy() for x in s.get()]
    t_g, _ = s.time()
    assert abs(t_g - t_o) <= TOL[precision] * t_o
    assert _state_rel(Wg, Wo) < TOL[precision], _state_rel(Wg, Wo)
    # gradients: relative to the largest gradient of each component
    for q in range(5):
        ref = dWo[3 * q:3 * q + 3]
        if np.abs(ref).max() > 1e-10:
            assert _rel(dWg[3 * q:3 * q + 3], ref) < TOL[precision], q


@pytest.mark.parametrize("precision", [0, 1])
def test_config1_sine_wave_ten_steps(cuda, oracle_mod, precision):
    """The 3072-cell density wave (8^3 hexes x 6, jitter 0.1, linear
    weights, full flux, CFL 0.5, 10 steps) in full."""
    mesh, W, dW = I.sine_wave_case(n=8)
    g = gks.Mesh(mesh)
    s = gks.State(g, gks.params(weno=0, cfl=0.5, precision=precision))
    s.init(W, dW)
    o = oracle_mod.Mesh(mesh)
    Wo, dWo, t_o, _ = o.run(oracle_mod.params(weno=0, cfl=0.5), W, dW, nsteps=10)
    s.step(10)
    s.sync()
    Wg, dWg = [x.cpu().numpy() for x in s.get()]
    assert _state_rel(Wg, Wo) < TOL[precision]
    for q in range(5):
        assert _rel(dWg[3 * q:3 * q + 3], dWo[3 * q:3 * q + 3]) < TOL[precision]
    # accuracy against the exact solution is the same in both precisions
    We, _ = I.sine_wave_state(mesh, t=t_o)
    vol = g.geometry()["vol"]
    l1_g = (vol * np.abs(Wg[0] - We[0])).sum() / vol.sum()
    l1_o = (vol * np.abs(Wo[0] - We[0])).sum() / vol.sum()
    assert abs(l1_g - l1_o) < 1e-3 * l1_o


def _grad_rel(dWg, dWo):
    """max over components with a gradient above 1e-10 of the normwise
    relative error of the gradient (its three directions share one scale)."""
    return max(_rel(dWg[3 * q:3 * q + 3], dWo[3 * q:3 * q + 3]) for q in range(5)
               if np.abs(dWo[3 * q:3 * q + 3]).max() > 1e-10)


@pytest.mark.parametrize("precision", [0, 1])
def test_config2_sod_full_size_three_steps(cuda, oracle_mod, precision):
    """The 24,576-cell Sod tube (64 x 8 x 8 hexes x 6, WENO) at full size,
    in the launch configuration the benchmark times (its autotuned variant
    included): three steps, every cell, averages and gradients."""
    mesh, W, dW = I.sod_case()
    g = gks.Mesh(mesh)
    assert (g.nc, g.nf, g.n_boundary) == (24576, 49280, 256)
    s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=precision))
    s.init(W, dW)
    s.autotune(steps=3, cache=False)  # restores the initial state
    o = oracle_mod.Mesh(mesh)
    Wo, dWo, to, _ = o.run(oracle_mod.params(weno=1, cfl=0.5), W, dW, nsteps=3)
    s.step(3)
    s.sync()
    Wg, dWg = [x.cpu().numpy() for x in s.get()]
    assert abs(s.time()[0] - to) <= TOL[precision] * to
    assert _state_rel(Wg, Wo) < TOL[precision], _state_rel(Wg, Wo)
    assert _grad_rel(dWg, dWo) < TOL[precision], _grad_rel(dWg, dWo)


_DEVELOPED = {}


def _developed_sod(oracle_mod):
    """The 36,864-cell Sod tube (96 x 8 x 8 hexes x 6) after three oracle
    steps from its seeded initial state, and the oracle's fourth step from
    there: the discontinuity has spread over a few cells and the
    reconstruction's second-derivative terms are at their largest."""
    if not _DEVELOPED:
        mesh, W, dW = I.sod_case(nx=96, nyz=8)
        om = oracle_mod.Mesh(mesh)
        p = oracle_mod.params(weno=1, cfl=0.5)
        W3, dW3, _, _ = om.run(p, W, dW, nsteps=3)
        dt = om.timestep(p, W3)
        W4, dW4, _ = om.step(p, W3, dW3, dt)
        _DEVELOPED.update(mesh=mesh, W3=W3, dW3=dW3, dt=dt, W4=W4, dW4=dW4)
    return _DEVELOPED


@pytest.mark.parametrize("precision,fused", [(0, 0), (1, 0), (1, 1), (2, 0)])
def test_sod_one_step_from_developed_discontinuity(cuda, oracle_mod, precision, fused):
    """One step from the oracle's state at step 3 of the Sod tube, with the
    oracle's step size, against the oracle's step 4: every cell, averages
    and gradients, at the tolerance of the precision (the FP32 bulk with
    either form of the stage).  This is the per-step parity at a sharp
    discontinuity; over several steps from the initial jump the FP32 forms
    drift from the FP64 result there by more than one step's rounding, as
    the nonlinear weights amplify it."""
    d = _developed_sod(oracle_mod)
    g = gks.Mesh(d["mesh"])
    s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=precision))
    if fused:
        s.set_fused(True)
    s.init(d["W3"], d["dW3"])
    s.step(1, d["dt"])
    s.sync()
    Wg, dWg = [x.cpu().numpy() for x in s.get()]
    # FP64: at the developed jump the reconstruction's second-derivative
    # coefficients reach ~6e3 times the state scale, and the 16-term operator
    # products cancel down to O(1) values, so a different rounding order moves
    # the result by ~16 x 6e3 x 2^-53 ~ 1e-11 per reconstruction; 5e-11 bounds
    # a step (two reconstructions and the flux built on them)
    tol = 5e-11 if precision == 0 else TOL[1]
    es, eg = _state_rel(Wg, d["W4"]), _grad_rel(dWg, d["dW4"])
    print("developed Sod, one step, precision %d fused %d: state %.3g gradient %.3g" % (precision, fused, es, eg))
    assert es < tol and eg < tol, (es, eg)


@pytest.mark.parametrize("precision", [0, 1])
def test_sod_tube_16x4x4_ten_steps(cuda, oracle_mod, precision):
    """WENO over ten steps on a Sod tube of 16 x 4 x 4 hexes x 6 (1,536
    cells, open x ends, y and z periodic): the shock, the contact and the
    rarefaction cross several cells, averages and gradients in full."""
    mesh = I.box_mesh((16, 4, 4), (1.0, 0.25, 0.25), (False, True, True), jitter=0.1, seed=51)
    W, dW = I.riemann_x_state(mesh)
    kw = dict(weno=1, cfl=0.5)
    g = gks.Mesh(mesh)
    s = gks.State(g, gks.params(precision=precision, **kw))
    s.init(W, dW)
    Wo, dWo, to, _ = oracle_mod.Mesh(mesh).run(oracle_mod.params(**kw), W, dW, nsteps=10)
    s.step(10)
    s.sync()
    Wg, dWg = [x.cpu().numpy() for x in s.get()]
    assert abs(s.time()[0] - to) <= TOL[precision] * to
    assert _state_rel(Wg, Wo) < TOL[precision], _state_rel(Wg, Wo)
    assert _grad_rel(dWg, dWo) < TOL[precision], _grad_rel(dWg, dWo)


@pytest.mark.parametrize("precision", [0, 1])
def test_density_wave_12_cubed_weno_ten_steps(cuda, oracle_mod, precision):
    """WENO over ten steps on the periodic density wave at 12^3 hexes x 6
    (10,368 cells): a smooth field, where the gradients are the most
    exposed to rounding (no jump sets their scale)."""
    mesh, W, dW = I.sine_wave_case(n=12)
    kw = dict(weno=1, cfl=0.5)
    g = gks.Mesh(mesh)
    s = gks.State(g, gks.params(precision=precision, **kw))
    s.init(W, dW)
    Wo, dWo, to, _ = oracle_mod.Mesh(mesh).run(oracle_mod.params(**kw), W, dW, nsteps=10)
    s.step(10)
    s.sync()
    Wg, dWg = [x.cpu().numpy() for x in s.get()]
    assert _state_rel(Wg, Wo) < TOL[precision], _state_rel(Wg, Wo)
    assert _grad_rel(dWg, dWo) < TOL[precision], _grad_rel(dWg, dWo)


@pytest.mark.parametrize("name", ["sod_small_weno", "sine_n3_weno", "closed_box_weno", "sine_n2_weno2"])
def test_fp64_operator_variant_parity(cuda, oracle_mod, name):
    """Precision 2 (FP32 bulk with the stencil operators, moments and their
    products in FP64): reconstruction and ten steps against the oracle at
    the FP32 tolerance, and within the same tolerance of precision 1."""
    mesh, W, dW, s, o, p = _setup(cuda, oracle_mod, name, 2)
    poly_g, slopes_g, fb_g = [x.cpu().numpy() for x in s.debug_reconstruct()]
    poly_o, slopes_o, fb_o = o.reconstruct(p, W, dW)
    np.testing.assert_array_equal(fb_g, fb_o)
    for q in range(5):
        for lo, hi in ((0, 1), (1, 4), (4, 10)):
            if np.abs(poly_o[:, q, lo:hi]).max() > 1e-12:
                assert _rel(poly_g[:, q, lo:hi], poly_o[:, q, lo:hi]) < TOL[1], (q, lo)
    nsteps = STEPS.get(name, 10)
    Wo, dWo, t_o, _ = o.run(p, W, dW, nsteps=nsteps)
    s.step(nsteps)
    s.sync()
    Wg, dWg = [x.cpu().numpy() for x in s.get()]
    assert _state_rel(Wg, Wo) < TOL[1], _state_rel(Wg, Wo)
    assert _grad_rel(dWg, dWo) < TOL[1], _grad_rel(dWg, dWo)


@pytest.mark.parametrize("precision", [1, 2])
def test_config2_sod_to_t_end_equal_l1(cuda, precision):
    """The full Sod tube to t = 0.2 (about 300 steps, every shock-tube wave
    well developed): the FP32-bulk runs stay within the FP32 tolerance of the
    FP64 run in density, and their L1 error against the exact Riemann
    solution equals the FP64 run's to three significant digits."""
    mesh, W, dW = I.sod_case()
    g = gks.Mesh(mesh)
    vol = g.geometry()["vol"]
    exact = None
    out = {}
    for prec in (0, precision):
        s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=prec))
        s.init(W, dW)
        t = s.run(t_end=0.2, chunk=64)
        Wg = s.get()[0].cpu().numpy()
        if exact is None:
            exact = I.riemann_x_exact_density(mesh, t)
        out[prec] = (Wg, (vol * np.abs(Wg[0] - exact)).sum() / vol.sum())
        del s
    (W64, l1_64), (W32, l1_32) = out[0], out[precision]
    assert abs(l1_32 - l1_64) < 1e-3 * l1_64, (l1_32, l1_64)
    assert np.abs(W32[0] - W64[0]).max() / np.abs(W64[0]).max() < 1e-3


def test_time_step_rule_and_t_end(cuda, oracle_mod):
    mesh, W, dW, s, o, p = _setup(cuda, oracle_mod, "sod_small_weno", 0)
    assert abs(s.timestep() - o.timestep(p, W)) <= 1e-14 * o.timestep(p, W)
    dt0 = o.timestep(p, W)
    t_end = 2.5 * dt0
    t = s.run(t_end=t_end, chunk=4)
    assert abs(t - t_end) < 1e-14
    # steps at t = t_end are no-ops
    Wa, _ = s.get()
    s.step(3, 0.0, t_end)
    s.sync()
    Wb, _ = s.get()
    assert cuda.equal(Wa, Wb)


def test_free_stream_and_conservation_on_gpu(cuda):
    mesh = I.box_mesh((4, 4, 4), jitter=0.1, seed=41)
    g = gks.Mesh(mesh)
    vol = g.geometry()["vol"]
    for precision in (0, 1):
        s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=precision))
        W = np.empty((5, g.nc))
        U = np.array([0.7, -0.2, 0.4])
        W[0], W[1:4], W[4] = 1.1, (1.1 * U)[:, None], 2.0 / 0.4 + 0.5 * 1.1 * U @ U
        s.init(W, np.zeros((15, g.nc)))
        s.step(5)
        s.sync()
        Wg, dWg = [x.cpu().numpy() for x in s.get()]
        tol = 1e-13 if precision == 0 else 1e-6
        assert np.abs(Wg - W).max() < tol * 5
        W2, dW2 = I.sine_wave_state(mesh)
        s.init(W2, dW2)
        s.step(5)
        s.sync()
        Wg, _ = [x.cpu().numpy() for x in s.get()]
        tot0, tot1 = (W2 * vol).sum(1), (Wg * vol).sum(1)
        ctol = 1e-13 if precision == 0 else 1e-7
        assert np.abs(tot1 - tot0).max() < ctol * np.abs(tot0).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_host_buffer_entry_point_matches_device_path(cuda, precision):
    mesh, W, dW = I.sine_wave_case(n=4)
    g = gks.Mesh(mesh)
    s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=precision))
    s.init(W, dW)
    s.step(3)
    s.sync()
    Wd, dWd = [x.cpu().numpy() for x in s.get()]
    Wh = cuda.tensor(W).pin_memory()
    dWh = cuda.tensor(dW).pin_memory()
    s2 = gks.State(g, gks.params(weno=1, cfl=0.5, precision=precision))
    s2.step_host(Wh, dWh, nsteps=3)
    np.testing.assert_array_equal(Wh.numpy(), Wd)
    np.testing.assert_array_equal(dWh.numpy(), dWd)


def test_bad_state_is_reported(cuda):
    """A cell with negative pressure: the step runs (NaN arithmetic only, no
    fault) and the device error flag surfaces as GKS_E_STATE."""
    mesh, W, dW = I.sine_wave_case(n=3)
    W = W.copy()
    W[4, 5] = -1.0
    g = gks.Mesh(mesh)
    s = gks.State(g, gks.params(weno=0, cfl=0.5))
    s.init(W, dW)
    s.step(1, dt_fixed=1e-3)
    with pytest.raises(gks.GksError) as e:
        s.sync()
    assert e.value.status == -4


def test_residual_matches_state_change(cuda):
    mesh, W, dW = I.sine_wave_case(n=3)
    g = gks.Mesh(mesh)
    s = gks.State(g, gks.params(weno=1, cfl=0.5))
    s.init(W, dW)
    s.step(2)
    s.sync()
    Wa, _ = s.get()
    s.step(1)
    s.sync()
    Wb, _ = s.get()
    _, dt = s.time()
    r = s.residual()
    ref = np.sqrt((((Wb - Wa).cpu().numpy() / dt) ** 2).mean(1))
    np.testing.assert_allclose(r, ref, rtol=1e-10)


def test_config4_vortex_full_size_one_step(cuda, oracle_mod):
    """The isentropic vortex (strength 5, free stream Ma 0.5 along the
    diagonal, periodic [0,10]^3) in the configuration the benchmark's adjoint
    leg runs: linear weights, CFL 0.5.  The recipe is checked against the
    oracle element by element on 16^3 hexes x 6 (24,576 cells), FP64 and
    FP32 bulk.  At full size (64^3 x 6 = 1,572,864 cells), where the oracle
    would take minutes, one step is checked by what holds at any size:
    Sum |Omega| W conserved to FP64 rounding in both precisions, and the FP32
    cell averages (momentum components on one shared scale) and gradients
    within 2e-5 of the FP64 path's, which matches the oracle at 1e-11 on the
    16^3 mesh."""
    kw = dict(weno=0, cfl=0.5)
    mesh, W, dW = I.isentropic_vortex_case(n=16, order=2)
    Wo, dWo, to, _ = oracle_mod.Mesh(mesh).run(oracle_mod.params(**kw), W, dW, nsteps=1)
    g = gks.Mesh(mesh)
    for precision in (0, 1):
        s = gks.State(g, gks.params(precision=precision, **kw))
        s.init(W, dW)
        s.step(1)
        s.sync()
        Wg, dWg = [x.cpu().numpy() for x in s.get()]
        assert abs(s.time()[0] - to) <= TOL[precision] * to
        assert _state_rel(Wg, Wo) < TOL[precision]
        for q in range(5):
            assert _rel(dWg[3 * q:3 * q + 3], dWo[3 * q:3 * q + 3]) < TOL[precision], q

    mesh, W, dW = I.isentropic_vortex_case(n=64, order=2)
    g = gks.Mesh(mesh)
    assert g.nc == 1572864
    geo = g.geometry()
    vol, dr = geo["vol"], geo["dr"]
    res = {}
    for precision in (0, 1):
        s = gks.State(g, gks.params(precision=precision, **kw))
        s.init(W, dW)
        s.step(1)
        s.sync()
        res[precision] = [x.cpu().numpy() for x in s.get()] + [s.time()[0]]
        del s
    total0 = W @ vol
    scale = (np.abs(W) @ vol).max()
    for precision, (Wg, _, _) in res.items():
        assert np.abs(Wg @ vol - total0).max() <= 1e-11 * scale, precision
    (W64, dW64, t64), (W32, dW32, t32) = res[0], res[1]
    assert abs(t32 - t64) <= TOL[1] * t64
    mom = np.abs(W64[1:4]).max()
    for q in range(5):
        sc = mom if 1 <= q <= 3 else np.abs(W64[q]).max()
        assert np.abs(W32[q] - W64[q]).max() < TOL[1] * sc, q
    assert _grad_rel(dW32, dW64) < TOL[1], _grad_rel(dW32, dW64)
