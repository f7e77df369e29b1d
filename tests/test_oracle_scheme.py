"""Whole-step pins of the oracle (Sec. 2.3, Sec. 3, Sec. 5): the S2O4 stage
algebra, free-stream preservation, discrete conservation, the divergence
theorem for the gradient update, the convergence order on smooth advection
and the Sod shock tube against its exact solution."""
import math

import numpy as np
import pytest

from paper_2102_01366_gb300 import inputs as I


@pytest.mark.parametrize("z", [0.4, 0.1, -0.25, -1.0])
def test_s2o4_reproduces_fourth_order_taylor(oracle_mod, z):
    """Eq. s2o4 with the linear flux fit of Eq. linear-system, on y' = lam y
    with a flux linear in time: one step is 1 + z + z^2/2 + z^3/6 + z^4/24."""
    got = oracle_mod.s2o4_linear_ode(z)
    assert abs(got - (1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24)) < 1e-15


@pytest.mark.parametrize("periodic", [(True, True, True), (False, True, True)])
@pytest.mark.parametrize("weno", [0, 1])
def test_free_stream_preserved(oracle_mod, periodic, weno):
    mesh = I.box_mesh((3, 3, 3), (1, 1, 1), periodic, jitter=0.1, seed=21)
    om = oracle_mod.Mesh(mesh)
    W = np.empty((5, om.nc))
    U = np.array([0.8, -0.3, 0.45])
    W[0], W[1:4], W[4] = 1.3, (1.3 * U)[:, None], 2.0 / 0.4 + 0.5 * 1.3 * U @ U
    dW = np.zeros((15, om.nc))
    W1, dW1, _, _ = om.run(oracle_mod.params(weno=weno), W, dW, nsteps=3)
    assert np.abs(W1 - W).max() < 1e-13
    assert np.abs(dW1).max() < 1e-12


@pytest.mark.parametrize("weno", [0, 1])
def test_conservation(oracle_mod, weno):
    mesh = I.box_mesh((3, 3, 3), jitter=0.1, seed=22)
    W, dW = I.sine_wave_state(mesh)
    om = oracle_mod.Mesh(mesh)
    vol = om.geometry()["vol"]
    W1, dW1, _, _ = om.run(oracle_mod.params(weno=weno), W, dW, nsteps=3)
    tot0 = (W * vol).sum(1)
    tot1 = (W1 * vol).sum(1)
    assert np.abs(tot1 - tot0).max() < 1e-14 * np.abs(tot0).max()
    # periodic box: the face sums of the divergence theorem cancel pairwise
    assert np.abs((dW1 * vol).sum(1)).max() < 1e-13
    assert np.abs(W1 - W).max() > 1e-3  # the state did move


def test_divergence_theorem_exact_for_linear_data(oracle_mod):
    """At t = 0 with linear data (reproduced exactly on both sides of every
    interior face), the interface value is the field itself, so the face
    sums of Eq. gauss-formula return the exact gradient in every cell that
    has no open-boundary face (there the ghost side is the cell average)."""
    mesh = I.box_mesh((5, 2, 2), (1.0, 0.4, 0.4), (False, True, True), jitter=0.1, seed=23)
    om = oracle_mod.Mesh(mesh)
    geo, top = om.geometry(), om.topology()
    b = 0.3
    W = np.zeros((5, om.nc))
    W[0] = 1.0 + b * geo["cen"][:, 0]
    W[4] = 2.5
    dW = np.zeros((15, om.nc))
    dW[0] = b
    rec = om.face_records(oracle_mod.params(), W, dW, 1e-3, 1)
    G0 = np.zeros((om.nc, 15))
    for c in range(om.nc):
        for f in range(4):
            G0[c] += top["csr_sign"][c, f] * rec[top["csr_face"][c, f], 25:40]
    G0 /= geo["vol"][:, None]
    expect = np.zeros((om.nc, 15))
    expect[:, 0] = b
    inner = (top["nbr"] >= 0).all(1)
    assert inner.sum() > 0.8 * om.nc
    np.testing.assert_allclose(G0[inner], expect[inner], atol=1e-13)


def _wave1d_state(mesh, t):
    def f(x):
        rho = 1 + 0.2 * np.sin(2 * np.pi * (x[..., 0] - t))
        dr = 0.2 * 2 * np.pi * np.cos(2 * np.pi * (x[..., 0] - t))
        z = np.zeros_like(rho)
        Wv = np.stack([rho, rho, z, z, 2.5 + 0.5 * rho], -1)
        dWv = np.zeros(rho.shape + (15,))
        for q, c in enumerate([1.0, 1.0, 0.0, 0.0, 0.5]):
            dWv[..., 3 * q] = c * dr
        return np.concatenate([Wv, dWv], -1)
    a = I.cell_average(mesh, f)
    return np.ascontiguousarray(a[:, :5].T), np.ascontiguousarray(a[:, 5:].T)


@pytest.mark.parametrize("weno,order,expect", [(0, 3, 2.6), (1, 3, 2.6), (1, 2, 1.7)])
def test_convergence_order_smooth_advection(oracle_mod, weno, order, expect):
    """A density wave along x (rho = 1 + 0.2 sin 2 pi (x - t), U = (1,0,0),
    p = 1) on jittered tetrahedral meshes nx x 2 x 2 of isotropic hexes;
    the L1 error of the density averages falls at the scheme's order (third
    order, Tables 1-2; second order for R^2nd, Table 3)."""
    errs = []
    for nx in (8, 16):
        h = 1.0 / nx
        mesh = I.box_mesh((nx, 2, 2), (1.0, 2 * h, 2 * h), (True, True, True), jitter=0.1, seed=3)
        om = oracle_mod.Mesh(mesh)
        W, dW = _wave1d_state(mesh, 0.0)
        W1, _, t, _ = om.run(oracle_mod.params(weno=weno, order=order, cfl=0.5), W, dW, t_end=0.05)
        We, _ = _wave1d_state(mesh, t)
        vol = om.geometry()["vol"]
        errs.append((vol * np.abs(W1[0] - We[0])).sum() / vol.sum())
    assert math.log2(errs[0] / errs[1]) > expect


def test_sod_against_exact_solution(oracle_mod):
    """Sod tube (WENO, CFL 0.5): the L1 density error against the exact
    Riemann solution falls under refinement and the density stays within
    the data's range up to 5e-3 (WENO is essentially, not strictly,
    non-oscillatory; 4e-3 is seen at these resolutions)."""
    errs = []
    for nx in (16, 32):
        mesh = I.box_mesh((nx, 2, 2), (1.0, 2.0 / nx, 2.0 / nx), (False, True, True), jitter=0.1, seed=6)
        W, dW = I.riemann_x_state(mesh)
        om = oracle_mod.Mesh(mesh)
        W1, _, t, _ = om.run(oracle_mod.params(weno=1, cfl=0.5), W, dW, t_end=0.1)
        exact = I.riemann_x_exact_density(mesh, t)
        vol = om.geometry()["vol"]
        errs.append((vol * np.abs(W1[0] - exact)).sum() / vol.sum())
        assert W1[0].max() < 1.0 + 5e-3 and W1[0].min() > 0.125 - 5e-3
    assert errs[1] < 0.8 * errs[0]


def _euler_flux(Wv, axis, gamma=1.4):
    rho = Wv[0]
    U = Wv[1:4] / rho
    p = (gamma - 1.0) * (Wv[4] - 0.5 * rho * U @ U)
    f = np.array([rho * U[axis], rho * U[0] * U[axis], rho * U[1] * U[axis], rho * U[2] * U[axis],
                  U[axis] * (Wv[4] + p)])
    f[1 + axis] += p
    return f


def _jacobian(Wv, axis, h=1e-6):
    return np.stack([(_euler_flux(Wv + h * e, axis) - _euler_flux(Wv - h * e, axis)) / (2 * h)
                     for e in np.eye(5)], axis=1)


def test_face_records_for_linear_field_in_global_frame(oracle_mod):
    """A linear field (every conservative variable affine in x), smooth
    solver, tau = 0: both sides reconstruct the field exactly, so at each
    Gauss point the flux is linear in time with F = F_n(W) and
    dF/dt = -J_n div F, and the interface state moves by -dt div F.  The
    face records, rotated back to the global frame, must equal the same
    quadrature of these closed forms.  This pins the frame matrix, the
    rotation of gradients into the face frame and back, the Gauss points
    and the record assembly."""
    mesh = I.box_mesh((4, 4, 4), (1.0, 1.0, 1.0), (False, False, False), jitter=0.1, seed=24)
    om = oracle_mod.Mesh(mesh)
    geo, top = om.geometry(), om.topology()
    W0 = np.array([1.0, 0.3, -0.2, 0.1, 2.5])
    G = np.array([[0.10, -0.05, 0.08],
                  [0.04, 0.07, -0.03],
                  [-0.06, 0.02, 0.05],
                  [0.03, -0.08, 0.02],
                  [0.09, 0.05, -0.07]])  # G[q, i] = d W_q / d x_i
    W = (W0[:, None] + G @ geo["cen"].T)
    dW = np.repeat(G.reshape(15, 1), om.nc, axis=1)
    dt = 2e-3
    p = oracle_mod.params(smooth_flux=1)
    rec1 = om.face_records(p, W, dW, dt, 1)
    rec2 = om.face_records(p, W, dW, dt, 2)
    good = (top["nbr"] >= 0).sum(1) >= 3
    checked = 0
    for f in range(om.nf):
        l, r = top["face_lr"][f]
        if l < 0 or r < 0 or not good[l] or not good[r]:
            continue  # open-boundary faces see the cell average on the ghost side
        c = l if l >= 0 else r
        X = (geo["gp_l"][f] if l >= 0 else geo["gp_r"][f]) + geo["cen"][c]
        n = geo["fnorm"][f]
        w = geo["farea"][f] / 3.0
        Fh = np.zeros(5)
        dG = np.zeros((5, 3))
        for k in range(3):
            Wk = W0 + G @ X[k]
            div = sum(_jacobian(Wk, a) @ G[:, a] for a in range(3))
            Fn = sum(n[a] * _euler_flux(Wk, a) for a in range(3))
            Jn = sum(n[a] * _jacobian(Wk, a) for a in range(3))
            Fh += w * (0.5 * dt * Fn - dt * dt / 8.0 * Jn @ div)
            dG += w * np.outer(-dt * div, n)
        np.testing.assert_allclose(rec1[f, 0:5], Fh, rtol=1e-8, atol=1e-12)
        np.testing.assert_allclose(rec2[f, 5:20], dG.reshape(15), rtol=1e-7, atol=1e-12)
        checked += 1
    assert checked > 0.7 * om.nf


def test_open_boundary_is_stable(oracle_mod):
    """Rounding-size noise on a uniform state next to open boundaries stays
    bounded (the ghost side is the interior average with zero gradient);
    copying the interior Gauss-point state instead grows it ~10^7-fold in
    100 steps."""
    nx = 16
    mesh = I.box_mesh((nx, 2, 2), (1.0, 2.0 / nx, 2.0 / nx), (False, True, True), jitter=0.1, seed=6)
    om = oracle_mod.Mesh(mesh)
    rng = np.random.default_rng(0)
    W0 = np.zeros((5, om.nc))
    W0[0], W0[4] = 1.0, 2.5
    W = W0 * (1 + 1e-7 * rng.standard_normal(W0.shape))
    W[1:4] = 1e-7 * rng.standard_normal((3, om.nc))
    W, dW, _, _ = om.run(oracle_mod.params(weno=1, cfl=0.5), W, np.zeros((15, om.nc)), nsteps=60)
    assert np.abs(W - W0).max() < 1e-3


@pytest.mark.parametrize("weno,viscous,smooth,prandtl,ends", [
    (0, 0, 0, 1.0, None), (0, 0, 1, 1.0, None), (0, 1, 0, 1.0, None), (0, 1, 1, 1.0, None), (0, 1, 0, 0.72, None),
    (1, 0, 0, 1.0, None), (1, 1, 0, 0.72, None), (0, 0, 0, 1.0, "open"), (1, 0, 0, 1.0, "slip"),
    (0, 1, 0, 1.0, "noslip"), (1, 1, 0, 0.72, "noslip"), (1, 0, 0, 1.0, "fixed"), (0, 1, 0, 1.0, "fixed"),
    (0, 0, 0, 1.0, "order2"), (1, 0, 0, 1.0, "order2"), (0, 0, 0, 1.0, "lowp"), (1, 0, 0, 1.0, "lowp"),
    (1, 1, 0, 0.72, "isothermal"), (1, 1, 0, 1.0, "moving")])
def test_torch_restatement_matches_the_oracle_step(oracle_mod, weno, viscous, smooth, prandtl, ends):
    """oracle/torch_step.py (the step in plain PyTorch CPU operations, for the
    autograd reverse sweep that checks the library's adjoint) reproduces the
    C oracle's step on a jittered mesh: linear or WENO weights, full or
    smooth flux, Euler or Navier-Stokes, with the Pr fix; periodic, or with
    open, slip-wall, non-slip-wall or fixed x ends."""
    import torch
    from oracle import torch_step as TS
    rng = np.random.Generator(np.random.PCG64(61))
    fixed = None
    order = 2 if ends == "order2" else 3
    if ends in (None, "order2", "lowp"):
        mesh = I.box_mesh((3, 3, 3), jitter=0.1, seed=61)
        W, dW = I.sine_wave_state(mesh, u=(0.8, 0.5, -0.3))
    else:
        mesh = I.box_mesh((4, 3, 3), (1.0, 0.75, 0.75), (False, True, True), jitter=0.1, seed=61)
        if ends != "open":
            kind = {"slip": I.BC_SLIP_WALL, "noslip": I.BC_NOSLIP_WALL, "fixed": I.BC_FIXED,
                    "isothermal": I.BC_ISOTHERMAL_WALL, "moving": I.BC_MOVING_WALL}[ends]
            mesh["bkind"] = I.boundary_kinds(mesh, {(0, "lo"): kind, (0, "hi"): kind})
        W, dW = I.sine_wave_state(mesh, k=8.0 * math.pi / 3.0, u=(0.6, 0.5, -0.3))
    W = W * (1.0 + 0.01 * rng.standard_normal(W.shape))
    dW = dW + 0.05 * rng.standard_normal(dW.shape)
    if ends == "lowp":  # a low-pressure cell whose reconstruction falls back to its average
        W[4, 0] = 0.5 * (W[1, 0] ** 2 + W[2, 0] ** 2 + W[3, 0] ** 2) / W[0, 0] + 0.05 / 0.4
    if ends == "fixed":
        fixed = (W * (1.0 + 0.02 * rng.standard_normal(W.shape)), 0.5 * dW)
        mesh["fixed_state"] = fixed
    o = oracle_mod.Mesh(mesh)
    kw = dict(mu=0.01 * viscous, viscous=viscous, smooth_flux=smooth, prandtl=prandtl, wall_temperature=0.9,
              wall_velocity=(0.0, 0.4, -0.2))
    p = oracle_mod.params(weno=weno, order=order, cfl=0.5, **kw)
    dt = 0.5 * o.timestep(p, W)
    Wo, dWo, _ = o.step(p, W, dW, dt)
    st = TS.Step(o, mu=kw["mu"], viscous=bool(viscous), smooth=bool(smooth), prandtl=prandtl, weno=bool(weno),
                 kinds=mesh.get("bkind"), fixed=fixed, order=order, wall_temperature=0.9,
                 wall_velocity=(0.0, 0.4, -0.2))
    Wt, dWt = st(torch.tensor(W), torch.tensor(dW), dt)
    assert bool(st.fallbacks[0].any()) == (ends == "lowp")
    for q in range(5):
        assert np.abs(Wt.numpy()[q] - Wo[q]).max() < 1e-14 * np.abs(Wo[q]).max()
        ref = dWo[3 * q:3 * q + 3]
        assert np.abs(dWt.numpy()[3 * q:3 * q + 3] - ref).max() < 1e-12 * np.abs(ref).max()
