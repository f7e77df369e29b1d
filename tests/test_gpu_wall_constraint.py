"""The constrained reconstruction at non-slip adiabatic walls (Sec. 4.4,
params.wall_constraint = 1) on the GPU path.  Element-by-element parity with
the oracle (reconstruction, face records, several steps, FP64 and FP32) is in
test_gpu_parity's constrained cases; here:

* the device's own output keeps the constraint: with linear weights the
  momenta of R vanish at the wall Gauss points (third order) or at the wall
  face centroids (second order), in both precisions;
* the FP32 bulk with FP64 operators (precision 2) against the oracle;
* the constrained operators follow the cells through the device orderings
  (bit-identical results) and the separate slopes pass, and the one-launch
  stage agrees with the separate kernels;
* the workspace grows only when the option is on and the mesh has such walls;
* the adjoint step, which does not differentiate the constrained stencils,
  rejects such a state instead of returning a wrong gradient.
"""
import math

import numpy as np
import pytest

from paper_2102_01366_gb300 import gks
from paper_2102_01366_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = {0: 1e-11, 1: 2e-5, 2: 2e-5}


@pytest.fixture(scope="module")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("these tests need a CUDA GPU")
    from paper_2102_01366_gb300 import _build
    _build.build()
    gks.lib()
    return torch


def _box(seed=61, nx=4):
    mesh = I.box_mesh((nx, 2, 2), (1.0, 0.5, 0.5), (False, True, True), jitter=0.1, seed=seed)
    mesh["bkind"] = I.boundary_kinds(mesh, {(0, "lo"): I.BC_NOSLIP_WALL, (0, "hi"): I.BC_NOSLIP_WALL})
    W, dW = I.sine_wave_state(mesh, k=4.0 * math.pi, u=(0.5, -0.3, 0.2))
    return mesh, W, dW


def _mono(P, X):
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    return (P[0] + P[1] * x + P[2] * y + P[3] * z + P[4] * x * x + P[5] * x * y + P[6] * x * z +
            P[7] * y * y + P[8] * y * z + P[9] * z * z)


def _rel_state(a, ref):
    mom = np.abs(ref[1:4]).max()
    out = 0.0
    for q in range(5):
        scale = mom if 1 <= q <= 3 else np.abs(ref[q]).max()
        out = max(out, np.abs(a[q] - ref[q]).max() / max(scale, 1e-300))
    return out


def _rel_grad(a, ref):
    mom = np.abs(ref[3:12]).max()
    out = 0.0
    for q in range(5):
        scale = mom if 1 <= q <= 3 else np.abs(ref[3 * q:3 * q + 3]).max()
        if scale > 1e-10:
            out = max(out, np.abs(a[3 * q:3 * q + 3] - ref[3 * q:3 * q + 3]).max() / scale)
    return out


def _wall_points(g, mesh, centroid):
    top, geo = g.topology(), g.geometry()
    out = {}
    for c in range(g.nc):
        pts = []
        for f in range(4):
            if top["nbr"][c, f] >= 0 or mesh["bkind"][c, f] != I.BC_NOSLIP_WALL:
                continue
            fi = top["csr_face"][c, f]
            gp = (geo["gp_l"][fi] if top["csr_sign"][c, f] > 0 else geo["gp_r"][fi]).reshape(3, 3)
            pts.append(gp.mean(axis=0, keepdims=True) if centroid else gp)
        if pts:
            out[c] = np.concatenate(pts)
    return out


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("order", [2, 3])
def test_device_momentum_vanishes_at_the_wall(cuda, precision, order):
    """Linear weights: R = P2 (order 3) of a wall cell's momenta is zero at
    its wall Gauss points, R = P1 (order 2) at its wall face centroids, to
    the rounding of the path's precision; without the option it is not."""
    mesh, W, dW = _box()
    g = gks.Mesh(mesh)
    pts = _wall_points(g, mesh, centroid=order == 2)
    assert len(pts) == 16  # 2 x 2 hexahedra on each wall, 2 tetrahedra each
    scale = np.abs(W[1:4]).max()
    worst = {}
    for wc in (1, 0):
        s = gks.State(g, gks.params(weno=0, order=order, cfl=0.5, precision=precision, wall_constraint=wc))
        s.init(W, dW)
        poly, _, fb = [x.cpu().numpy() for x in s.debug_reconstruct()]
        worst[wc] = max(np.abs(_mono(poly[c, q], X)).max() for c, X in pts.items() for q in (1, 2, 3))
        assert not fb.any()
    assert worst[1] < (1e-12 if precision == 0 else 2e-5) * scale, worst
    assert worst[0] > 1e-2 * scale, worst


@pytest.mark.parametrize("weno", [0, 1])
def test_fp64_operators_against_the_oracle(cuda, oracle_mod, weno):
    """Precision 2 (FP32 bulk, FP64 stencil operators, here also the
    constrained ones): five steps of the walled box against the oracle."""
    mesh, W, dW = _box(seed=62)
    kw = dict(weno=weno, cfl=0.5, viscous=1, mu=0.01, wall_constraint=1)
    g = gks.Mesh(mesh)
    s = gks.State(g, gks.params(precision=2, **kw))
    s.init(W, dW)
    s.step(5)
    s.sync()
    Wg, dWg = [x.cpu().numpy() for x in s.get()]
    Wo, dWo, to, _ = oracle_mod.Mesh(mesh).run(oracle_mod.params(**kw), W, dW, nsteps=5)
    assert abs(s.time()[0] - to) <= TOL[2] * to
    assert _rel_state(Wg, Wo) < TOL[2], _rel_state(Wg, Wo)
    assert _rel_grad(dWg, dWo) < TOL[2], _rel_grad(dWg, dWo)


@pytest.mark.parametrize("precision", [1, 2])
def test_orderings_and_slopes_pass_are_bit_identical(cuda, precision):
    """The constrained operators are uploaded in device-cell order, so every
    device ordering, either face order and the separate slopes pass give the
    same results to the bit."""
    mesh, W, dW = _box(seed=63)
    g = gks.Mesh(mesh)
    ref = None
    for order in (0, 1, 2):
        for variant in ((0, 3, 0), (1, 3, 1)):
            s = gks.State(g, gks.params(weno=1, cfl=0.5, viscous=1, mu=0.01, precision=precision,
                                        wall_constraint=1))
            s.set_cell_order(order)
            s.set_variant(*variant)
            s.init(W, dW)
            s.step(3)
            s.sync()
            out = [x.cpu() for x in s.get()] + [x.cpu() for x in s.debug_reconstruct()]
            if ref is None:
                ref = out
            else:
                for a, b in zip(ref, out):
                    assert cuda.equal(a, b), (order, variant)


def test_fused_stage_with_constrained_walls(cuda):
    """The one-launch stage (which always carries the wall path) against the
    separate kernels, FP32, three steps of the walled box."""
    mesh, W, dW = _box(seed=64)
    g = gks.Mesh(mesh)
    out = {}
    for fused in (0, 1):
        s = gks.State(g, gks.params(weno=1, cfl=0.5, viscous=1, mu=0.01, precision=1, wall_constraint=1))
        s.set_fused(fused)
        s.init(W, dW)
        s.step(3)
        s.sync()
        out[fused] = [x.cpu().numpy() for x in s.get()]
    assert _rel_state(out[1][0], out[0][0]) < 1e-6
    assert _rel_grad(out[1][1], out[0][1]) < 1e-5


def test_adjoint_rejects_the_constrained_stencils(cuda):
    import torch
    mesh, W, dW = _box(seed=65)
    g = gks.Mesh(mesh)
    s = gks.State(g, gks.params(weno=1, cfl=0.5, viscous=1, mu=0.01, precision=0, wall_constraint=1))
    s.init(W, dW)
    dt = s.timestep()
    Wt, dWt = torch.tensor(W, device="cuda"), torch.tensor(dW, device="cuda")
    with pytest.raises(gks.GksError) as e:
        s.adjoint_step(Wt, dWt, torch.ones_like(Wt), torch.zeros_like(dWt), dt)
    assert e.value.status == -8  # GKS_E_UNSUPPORTED
    # without the option the same state has an adjoint
    s0 = gks.State(g, gks.params(weno=1, cfl=0.5, viscous=1, mu=0.01, precision=0))
    s0.init(W, dW)
    lw, ldw = s0.adjoint_step(Wt, dWt, torch.ones_like(Wt), torch.zeros_like(dWt), dt)
    assert torch.isfinite(lw).all()
