"""Slip walls and the paper's one-dimensional problems (Sec. 4.4, Sec. 5.2)
on the GPU path.  Element-by-element parity with the oracle on walled meshes
is in test_gpu_parity (the closed-box and wall-reflection cases); here the
full-size workloads: the wall reflection against its exact solution in both
precisions, closed-box conservation, and the Shu-Osher and blast-wave runs
to the paper's end times with physical checks (undisturbed region, shock
position, peak density, positivity)."""
import math

import numpy as np
import pytest

from paper_2102_01366_gb300 import gks
from paper_2102_01366_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")
    from paper_2102_01366_gb300 import _build
    _build.build()
    gks.lib()
    return torch


def _run(mesh, W, dW, t_end, precision, **kw):
    g = gks.Mesh(mesh)
    s = gks.State(g, gks.params(precision=precision, **kw))
    s.init(W, dW)
    t = s.run(t_end=t_end)
    Wg, dWg = [x.cpu().numpy() for x in s.get()]
    return g, Wg, dWg, t


@pytest.fixture(scope="module")
def wall_reflection(cuda):
    mesh, W, dW = I.wall_reflection_case(nx=64, nyz=4)
    exact = I.wall_reflection_exact_density(mesh, 0.25)
    vol = gks.Mesh(mesh).geometry()["vol"]
    out = {}
    for precision in (0, 1):
        _, Wg, _, t = _run(mesh, W, dW, 0.25, precision, weno=1, cfl=0.5)
        assert abs(t - 0.25) < 1e-12
        out[precision] = (float((np.abs(Wg[0] - exact) * vol).sum() / vol.sum()), Wg)
    return out


def test_wall_reflection_matches_exact_solution(wall_reflection):
    """64 cells across (24,576 tets): L1(rho) below the oracle's 32-cell
    value (0.0167 on the thinner 32 x 2 x 2 mesh), and the two precisions
    give the same error to 3 digits."""
    l1_fp64, l1_fp32 = wall_reflection[0][0], wall_reflection[1][0]
    assert l1_fp64 < 0.0167, l1_fp64
    assert abs(l1_fp32 - l1_fp64) < 1e-3 * l1_fp64, (l1_fp32, l1_fp64)


@pytest.mark.parametrize("precision", [0, 1])
def test_closed_box_conserves(cuda, precision):
    mesh = I.box_mesh((16, 4, 4), (1.0, 0.25, 0.25), (False, True, True), jitter=0.1, seed=41)
    mesh["bkind"] = I.wall_kinds(mesh, (0,))
    W, dW = I.sine_wave_state(mesh, k=8.0 * math.pi, u=(0.7, 0.2, -0.1))
    g = gks.Mesh(mesh)
    vol = g.geometry()["vol"]
    s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=precision))
    s.init(W, dW)
    s.step(40)
    s.sync()
    W1 = s.get()[0].cpu().numpy()
    tot0, tot1 = (W * vol).sum(1), (W1 * vol).sum(1)
    tol = 1e-13 if precision == 0 else 1e-6
    for q in (0, 2, 3, 4):
        assert abs(tot1[q] - tot0[q]) < tol * np.abs(tot0).max(), q


@pytest.mark.parametrize("precision", [0, 1])
def test_fixed_ends_keep_a_stationary_contact(cuda, precision):
    """A linear density profile at rest under uniform pressure between two
    fixed boundaries is an exact steady state that the scheme keeps to
    round-off (the oracle pin of the same property, here at 12,288 cells)."""
    mesh = I.box_mesh((32, 4, 4), (1.0, 0.125, 0.125), (False, True, True), jitter=0.1, seed=42)
    mesh["bkind"] = I.boundary_kinds(mesh, {(0, "lo"): I.BC_FIXED, (0, "hi"): I.BC_FIXED})

    def lin(x):
        rho = 1.0 + 0.3 * x[..., 0]
        z = np.zeros_like(rho)
        return np.stack([rho, z, z, z, np.full_like(rho, 1.0 / 0.4)], axis=-1)
    W = I.cell_average(mesh, lin, order=3).T.copy()
    dW = np.zeros((15, W.shape[1]))
    dW[0] = 0.3
    g = gks.Mesh(mesh)
    s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=precision))
    s.init(W, dW)
    s.step(20)
    s.sync()
    W1 = s.get()[0].cpu().numpy()
    tol = 1e-13 if precision == 0 else 2e-5  # FP32: rounding of 20 steps
    assert np.abs(W1 - W).max() < tol * np.abs(W).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_shear_wave_between_noslip_walls(cuda, precision):
    """Viscous shear wave v = A sin(pi x) between non-slip adiabatic walls,
    32 cells across (24,576 tets), mu = 0.002, to t = 2: the decrement of the
    amplitude matches nu pi^2 t to 0.2 % (the oracle's 8-cell run: 1 %), mass
    and total energy are conserved (impermeable, adiabatic walls at rest)."""
    mesh, W, dW = I.shear_decay_case(nx=32, nyz=4)
    g, Wg, _, t = _run(mesh, W, dW, 2.0, precision, weno=1, cfl=0.5, viscous=1, mu=0.002)
    assert abs(t - 2.0) < 1e-12
    vol = g.geometry()["vol"]
    A0 = I.shear_decay_amplitude(mesh, W, vol=vol)
    A1 = I.shear_decay_amplitude(mesh, Wg, vol=vol)
    exact = A0 * math.exp(-0.002 * math.pi ** 2 * 2.0)
    assert abs(A1 - exact) < 2e-3 * (A0 - exact), (A0, A1, exact)
    tol = 1e-12 if precision == 0 else 1e-6
    for q in (0, 4):
        assert abs((Wg[q] * vol).sum() - (W[q] * vol).sum()) < tol * abs((W[q] * vol).sum()), q


@pytest.mark.parametrize("precision", [0, 1])
def test_shu_osher(cuda, precision):
    """Sec. 5.2 (a), 6 x 200 x 2 x 2 cells, third order, to t = 1.8.  The
    Mach-3 shock (speed 3.549 into the gas at rest) sits near x = 7.39; ahead
    of it the stationary entropy wave is undisturbed; behind it the inflow
    state holds at the left end; no negative density or pressure.  (The
    second-order scheme develops cell-to-cell noise behind the shock on this
    mesh and fails near t = 1.2-1.4.)"""
    mesh, W, dW = I.shu_osher_case(nx=200, nyz=2)
    g, Wg, _, t = _run(mesh, W, dW, 1.8, precision, weno=1, order=3, cfl=0.5)
    assert abs(t - 1.8) < 1e-12
    x = g.geometry()["cen"][:, 0]
    rho = Wg[0]
    # the flow is one-dimensional: the tetrahedra of the thin periodic cross
    # section imprint a transverse velocity of about 0.2-0.35 behind the Mach-3
    # shock; a transverse instability of that layer (seeded by rounding, it
    # reached 0.74 in an FP32 build with approximate division in the update
    # and smeared the shock) stays out
    assert np.abs(Wg[2:4] / rho).max() < 0.5, np.abs(Wg[2:4] / rho).max()
    ahead = x > 7.8
    assert np.abs(rho[ahead] - W[0][ahead]).max() < 2e-3
    assert abs(rho[x < 0.5].mean() - 3.857134) < 1e-3
    jump = np.abs(np.diff(rho[np.argsort(x)]))
    xs = np.sort(x)
    shock_x = xs[np.argmax(jump * (xs[1:] > 6.0))]
    assert 7.2 < shock_x < 7.6, shock_x
    assert 4.4 < rho.max() < 5.0, rho.max()


def test_blast_wave(cuda):
    """Sec. 5.2 (b), 6 x 200 x 2 x 2 cells with reflecting ends, to
    t = 0.038, third order, FP64, CFL 0.1 (about 17,000 steps).  Both blast
    waves have reflected and collided: the density peak of the collision
    (about 6 in converged solutions) lies near x = 0.78; mass and energy are
    conserved between the walls; the run stays positive.  The paper gives no
    CFL for this case; at CFL >= 0.15 the first step already drives a cell
    next to the 1000 : 0.01 pressure jump negative (the oracle agrees), and
    the FP32 and second-order runs at CFL 0.1 fail later: the scheme has no
    positivity limiter on cell averages."""
    mesh, W, dW = I.blast_wave_case(nx=200, nyz=2)
    precision = 0
    g, Wg, _, t = _run(mesh, W, dW, 0.038, precision, weno=1, order=3, cfl=0.1)
    assert abs(t - 0.038) < 1e-12
    geo = g.geometry()
    x, vol = geo["cen"][:, 0], geo["vol"]
    rho = Wg[0]
    assert rho.min() > 0.0
    tol = 1e-12 if precision == 0 else 1e-5
    for q in (0, 4):
        assert abs((Wg[q] * vol).sum() - (W[q] * vol).sum()) < tol * abs((W[q] * vol).sum()), q
    assert 5.0 < rho.max() < 7.0, rho.max()
    assert 0.75 < x[np.argmax(rho)] < 0.81, x[np.argmax(rho)]


def test_sphere_full_size_first_steps(cuda):
    """The 7,004,160-cell sphere shell in the configuration the benchmark
    times (WENO, viscous, Pr 0.72, from the free stream), FP64 and FP32 bulk,
    2 steps, checked through properties that hold at any size: cells whose
    stencils see only the free stream keep it (free-stream preservation on
    the curved, stretched shell: after 2 steps everything beyond r = 1 is
    untouched), mass is conserved (no mass crosses the non-slip wall, and the
    far-field faces carry the uniform free-stream flux, which sums to zero
    over the closed outer sphere), and the two precisions agree."""
    mesh, W, dW, mu = I.sphere_case()
    g = gks.Mesh(mesh)
    assert (g.nc, g.nf, g.n_boundary, g.n_singular) == (7004160, 14044800, 72960, 0)
    geo = g.geometry()
    vol, r = geo["vol"], np.linalg.norm(geo["cen"], axis=1)
    far = r > 1.0
    mass0 = (vol * W[0]).sum()
    out = {}
    for precision in (0, 1):
        s = gks.State(g, gks.params(precision=precision, weno=1, cfl=0.5, viscous=1, mu=mu, prandtl=0.72))
        s.init(W, dW)
        s.step(2)
        s.sync()
        Wg = s.get()[0].cpu().numpy()
        assert np.isfinite(Wg).all()
        scale = np.array([1.0, 0.2, 0.2, 0.2, W[4, 0]])[:, None]
        near_wall = np.abs(Wg - W)[:, ~far] / scale
        assert near_wall.max() > 1e-4  # the wall has started the flow
        tol = 1e-13 if precision == 0 else 1e-6
        assert (np.abs(Wg - W)[:, far] / scale).max() < tol
        assert abs((vol * Wg[0]).sum() - mass0) < (1e-13 if precision == 0 else 1e-7) * mass0
        out[precision] = Wg
        del s
    # FP32 bulk against FP64: the pole wedges next to the wall (30 times
    # thinner azimuthally than radially) carry the largest difference, ~1e-5
    # of the free-stream momentum after 2-3 steps
    scale = np.array([1.0, 0.2, 0.2, 0.2, W[4, 0]])[:, None]
    assert (np.abs(out[1] - out[0]) / scale).max() < 5e-5
