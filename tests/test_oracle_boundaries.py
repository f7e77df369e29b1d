"""Boundary faces in the oracle.

Slip walls (Sec. 4.4), pinned by what the mirror image
across a wall fixes independently of the oracle's formulas: no mass, energy
or tangential momentum crosses a wall (the ghost is the exact mirror of the
interior state at every Gauss point), a gas at rest in a closed box stays at
rest, a closed box conserves mass, energy and the tangential momenta, and a
gas moving between two walls reproduces the exact reflected-shock /
wall-rarefaction solution (each wave the Riemann problem between the gas and
its mirror image) with an error that falls under refinement.

Fixed boundaries (a prescribed state carried past the boundary: the
Shu-Osher right end of Sec. 5.2, a far field), pinned by a stationary
contact: a linear density profile at rest under uniform pressure is an exact
steady solution that the scheme reproduces to round-off when the ghost holds
the profile's value and gradient at each Gauss point, and visibly does not
with open ends."""
import math

import numpy as np
import pytest

from paper_2102_01366_gb300 import inputs as I


def _closed_box(nx=4, nyz=2, seed=31):
    mesh = I.box_mesh((nx, nyz, nyz), (1.0, 0.5, 0.5), (False, True, True), jitter=0.1, seed=seed)
    mesh["bkind"] = I.wall_kinds(mesh, (0,))
    return mesh


def _smooth_state(mesh, u=(0.6, -0.3, 0.2)):
    """Density wave on a moving gas, with cell-averaged gradients."""
    W, dW = I.sine_wave_state(mesh, amp=0.2, k=4.0 * np.pi, u=u, p=1.0)  # period 0.5 in y, z
    return W, dW


def test_wall_kinds_mark_the_end_planes(oracle_mod):
    mesh = _closed_box(nx=4, nyz=3)
    kind = mesh["bkind"]
    # every end-plane quad is two triangles, on both ends
    assert kind.sum() == 2 * 2 * 3 * 3
    om = oracle_mod.Mesh(mesh)
    top = om.topology()
    # walls only where the cell has no neighbour
    assert (top["nbr"][kind == 1] < 0).all()
    assert ((top["nbr"] < 0) == (kind == 1)).all()
    bad = kind.copy()
    bad[kind == 1] = 7
    with pytest.raises(ValueError):
        om.set_boundary(bad)


@pytest.mark.parametrize("stage", [1, 2])
@pytest.mark.parametrize("weno", [0, 1])
def test_no_mass_energy_or_tangential_momentum_through_a_wall(oracle_mod, stage, weno):
    mesh = _closed_box()
    W, dW = _smooth_state(mesh)
    om = oracle_mod.Mesh(mesh)
    top, geo = om.topology(), om.geometry()
    rec = om.face_records(oracle_mod.params(weno=weno), W, dW, 2e-3, stage)
    wall = (top["face_lr"] < 0).any(axis=1)
    assert wall.sum() == 2 * 2 * 2 * 2
    n = geo["fnorm"][wall]
    r = rec[wall]
    scale = np.abs(rec[:, :5]).max()
    # stage 1: entries 0-4 and 5-9 are fluxes; stage 2: entries 0-4
    blocks = (0, 5) if stage == 1 else (0,)
    for b in blocks:
        F = r[:, b:b + 5]
        assert np.abs(F[:, 0]).max() < 1e-14 * scale  # mass
        assert np.abs(F[:, 4]).max() < 1e-14 * scale  # energy
        mom = F[:, 1:4]
        tang = mom - (mom * n).sum(1)[:, None] * n
        assert np.abs(tang).max() < 1e-14 * scale
        assert np.abs((mom * n).sum(1)).min() > 1e-6 * scale  # the wall does push


def test_gas_at_rest_in_a_closed_box_stays_at_rest(oracle_mod):
    mesh = _closed_box()
    om = oracle_mod.Mesh(mesh)
    W = np.zeros((5, om.nc))
    W[0], W[4] = 1.2, 0.9 / 0.4
    dW = np.zeros((15, om.nc))
    W1, dW1, _, _ = om.run(oracle_mod.params(weno=1, cfl=0.5), W, dW, nsteps=4)
    assert np.abs(W1 - W).max() < 1e-13
    assert np.abs(dW1).max() < 1e-11


@pytest.mark.parametrize("order", [3, 2])
def test_closed_box_conservation(oracle_mod, order):
    mesh = _closed_box()
    W, dW = _smooth_state(mesh)
    om = oracle_mod.Mesh(mesh)
    vol = om.geometry()["vol"]
    W1, _, _, _ = om.run(oracle_mod.params(weno=1, order=order, cfl=0.5), W, dW, nsteps=4)
    tot0, tot1 = (W * vol).sum(1), (W1 * vol).sum(1)
    scale = np.abs(tot0).max()
    for q in (0, 2, 3, 4):  # mass, tangential momenta, energy
        assert abs(tot1[q] - tot0[q]) < 1e-14 * scale, q
    # the walls change the normal momentum
    assert abs(tot1[1] - tot0[1]) > 1e-4 * scale


def test_wall_reflection_against_exact_solution(oracle_mod):
    """(rho, u, p) = (1, 1, 1) between walls at x = 0 and 1 until t = 0.15:
    rarefaction at the left wall, reflected shock at the right wall (the
    waves meet only at t ~ 0.33).  L1(rho) falls with refinement (0.0209 and
    0.0144 at 12 and 24 cells across); a ghost that did not reflect leaves
    an error of order 0.1 in the shocked region alone."""
    l1 = []
    for nx in (12, 24):
        mesh, W, dW = I.wall_reflection_case(nx=nx, nyz=2)
        om = oracle_mod.Mesh(mesh)
        vol = om.geometry()["vol"]
        W1, _, t, _ = om.run(oracle_mod.params(weno=1, cfl=0.5), W, dW, t_end=0.15)
        assert abs(t - 0.15) < 1e-14
        exact = I.wall_reflection_exact_density(mesh, 0.15)
        l1.append(float((np.abs(W1[0] - exact) * vol).sum() / vol.sum()))
    assert l1[0] < 0.03, l1
    assert l1[1] < 0.8 * l1[0], l1


def _contact(seed=51):
    mesh = I.box_mesh((6, 2, 2), (1.0, 1 / 3, 1 / 3), (False, True, True), jitter=0.1, seed=seed)

    def lin(x):
        rho = 1.0 + 0.3 * x[..., 0]
        z = np.zeros_like(rho)
        return np.stack([rho, z, z, z, np.full_like(rho, 1.0 / 0.4)], axis=-1)
    W = I.cell_average(mesh, lin, order=3).T.copy()
    dW = np.zeros((15, W.shape[1]))
    dW[0] = 0.3
    return mesh, W, dW


@pytest.mark.parametrize("weno", [0, 1])
def test_fixed_boundary_keeps_a_stationary_contact(oracle_mod, weno):
    mesh, W, dW = _contact()
    change = {}
    for kind in (I.BC_OPEN, I.BC_FIXED):
        m = dict(mesh)
        m["bkind"] = I.boundary_kinds(mesh, {(0, "lo"): kind, (0, "hi"): kind})
        m["fixed_state"] = (W, dW)
        om = oracle_mod.Mesh(m)
        W1, dW1, _, _ = om.run(oracle_mod.params(weno=weno, cfl=0.5), W, dW, nsteps=3)
        change[kind] = (np.abs(W1 - W).max(), np.abs(dW1 - dW).max())
    assert change[I.BC_FIXED][0] < 1e-14 and change[I.BC_FIXED][1] < 1e-12, change
    assert change[I.BC_OPEN][0] > 1e-3, change


def test_uniform_flow_through_fixed_boundaries(oracle_mod):
    mesh = I.box_mesh((4, 2, 2), (1.0, 0.5, 0.5), (False, True, True), jitter=0.1, seed=52)
    mesh["bkind"] = I.boundary_kinds(mesh, {(0, "lo"): I.BC_FIXED, (0, "hi"): I.BC_FIXED})
    W, dW = I.riemann_x_state(mesh, left=(1.2, 1.5, 0.8), right=(1.2, 1.5, 0.8))
    mesh["fixed_state"] = (W, dW)
    om = oracle_mod.Mesh(mesh)
    W1, dW1, _, _ = om.run(oracle_mod.params(weno=1, cfl=0.5), W, dW, nsteps=3)
    assert np.abs(W1 - W).max() < 1e-13
    assert np.abs(dW1).max() < 1e-11


def test_fixed_boundary_needs_its_state(oracle_mod):
    mesh, W, dW = _contact()
    mesh["bkind"] = I.boundary_kinds(mesh, {(0, "hi"): I.BC_FIXED})
    om = oracle_mod.Mesh(mesh)
    with pytest.raises(ValueError):
        om.step(oracle_mod.params(weno=1), W, dW)


# ---------------------------------------------------------------- no-slip --
# Non-slip adiabatic walls at rest (Sec. 4.4): the ghost is the interior
# state reflected through the Gauss point with the velocity reversed, so the
# interface distribution carries no mass and no energy through the wall
# while the viscous solver supplies the wall shear.  Pinned by those fluxes,
# exact conservation of mass and energy in a closed box, and the decay rate
# of a viscous shear wave between two walls (v = A sin(pi x) e^{-nu pi^2 t}).

def _noslip_box(nx=4, nyz=2, seed=33):
    mesh = I.box_mesh((nx, nyz, nyz), (1.0, 0.5, 0.5), (False, True, True), jitter=0.1, seed=seed)
    mesh["bkind"] = I.boundary_kinds(mesh, {(0, "lo"): I.BC_NOSLIP_WALL, (0, "hi"): I.BC_NOSLIP_WALL})
    return mesh


@pytest.mark.parametrize("stage", [1, 2])
@pytest.mark.parametrize("viscous", [0, 1])
def test_no_mass_or_energy_through_a_noslip_wall(oracle_mod, stage, viscous):
    mesh = _noslip_box()
    W, dW = _smooth_state(mesh)
    om = oracle_mod.Mesh(mesh)
    top = om.topology()
    rec = om.face_records(oracle_mod.params(weno=1, viscous=viscous, mu=0.01), W, dW, 2e-3, stage)
    wall = (top["face_lr"] < 0).any(axis=1)
    scale = np.abs(rec[:, :5]).max()
    for b in ((0, 5) if stage == 1 else (0,)):
        F = rec[wall, b:b + 5]
        assert np.abs(F[:, 0]).max() < 1e-14 * scale  # mass
        assert np.abs(F[:, 4]).max() < 1e-14 * scale  # energy


def test_noslip_closed_box_conserves_mass_and_energy(oracle_mod):
    mesh = _noslip_box()
    W, dW = _smooth_state(mesh)
    om = oracle_mod.Mesh(mesh)
    vol = om.geometry()["vol"]
    W1, _, _, _ = om.run(oracle_mod.params(weno=1, cfl=0.5, viscous=1, mu=0.01), W, dW, nsteps=4)
    tot0, tot1 = (W * vol).sum(1), (W1 * vol).sum(1)
    for q in (0, 4):
        assert abs(tot1[q] - tot0[q]) < 1e-14 * abs(tot0[q]), q
    # the walls take momentum out (shear and pressure)
    assert np.abs(tot1[1:4] - tot0[1:4]).max() > 1e-6


def test_shear_wave_decays_at_the_viscous_rate(oracle_mod):
    """8 cells across, mu = 0.002 (mean free path ~ 2e-3 of the gap, so the
    BGK gas is in the Navier-Stokes regime), t = 2: the amplitude falls by
    3.9 %, and the computed decrement matches nu pi^2 t to 1 %; the inviscid
    solver keeps nearly all of the amplitude."""
    mesh, W, dW = I.shear_decay_case(nx=8, nyz=2)
    om = oracle_mod.Mesh(mesh)
    vol = om.geometry()["vol"]
    A0 = I.shear_decay_amplitude(mesh, W, vol=vol)
    exact = A0 * math.exp(-0.002 * math.pi ** 2 * 2.0)
    W1, _, t, _ = om.run(oracle_mod.params(weno=1, cfl=0.5, viscous=1, mu=0.002), W, dW, t_end=2.0)
    A1 = I.shear_decay_amplitude(mesh, W1, vol=vol)
    assert abs(A1 - exact) < 0.01 * (A0 - exact), (A0, A1, exact)
    W2, _, _, _ = om.run(oracle_mod.params(weno=1, cfl=0.5), W, dW, t_end=2.0)
    A2 = I.shear_decay_amplitude(mesh, W2, vol=vol)
    assert A2 - exact > 0.5 * (A0 - exact), (A0, A2, exact)


def _isothermal_box(nx=4, nyz=2, seed=40):
    mesh = I.box_mesh((nx, nyz, nyz), (1.0, 0.5, 0.5), (False, True, True), jitter=0.1, seed=seed)
    mesh["bkind"] = I.boundary_kinds(mesh, {(0, "lo"): I.BC_ISOTHERMAL_WALL, (0, "hi"): I.BC_ISOTHERMAL_WALL})
    return mesh


def _gas_at_rest(mesh, rho, p=1.0):
    nc = mesh["tet"].shape[0]
    W = np.zeros((5, nc))
    W[0], W[4] = rho, p / 0.4
    return W, np.zeros((15, nc))


def test_isothermal_wall_at_the_gas_temperature_keeps_it_at_rest(oracle_mod):
    """Sec. 4.4 non-slip isothermal wall: gas at rest whose temperature
    p / rho equals the wall's is an equilibrium (the ghost is the interior
    state), so it stays at rest."""
    mesh = _isothermal_box()
    W, dW = _gas_at_rest(mesh, rho=1.25)  # T = 0.8
    om = oracle_mod.Mesh(mesh)
    W1, dW1, _, _ = om.run(oracle_mod.params(weno=1, cfl=0.5, viscous=1, mu=0.01, wall_temperature=0.8), W, dW,
                           nsteps=5)
    assert np.abs(W1 - W).max() < 1e-13
    assert np.abs(dW1).max() < 1e-12


@pytest.mark.parametrize("t_gas,sign", [(1.2, -1.0), (0.8, 1.0)])
def test_isothermal_wall_heat_flows_from_hot_to_cold(oracle_mod, t_gas, sign):
    """Gas at rest at temperature t_gas between isothermal walls at T_w = 1,
    Navier-Stokes solver: the walls take heat from hotter gas and give it to
    colder gas (the total energy falls or rises), and the gas next to the
    walls moves toward the wall temperature while the middle has not yet
    felt it.  (The wall's heat flux is a viscous effect: with the Euler
    solver the isothermal ghost has no physical meaning.)"""
    mesh = _isothermal_box(nx=6)
    W, dW = _gas_at_rest(mesh, rho=1.0 / t_gas)
    om = oracle_mod.Mesh(mesh)
    geo = om.geometry()
    vol, cen = geo["vol"], geo["cen"][:, 0]
    p = oracle_mod.params(weno=1, cfl=0.5, viscous=1, mu=0.02, wall_temperature=1.0)
    W1, _, _, _ = om.run(p, W, dW, nsteps=6)
    assert sign * ((vol * W1[4]).sum() - (vol * W[4]).sum()) > 1e-3
    T1 = 0.4 * (W1[4] - 0.5 * (W1[1:4] ** 2).sum(0) / W1[0]) / W1[0]
    near = np.minimum(cen, 1.0 - cen) < 1.0 / 6.0
    assert sign * (T1[near].mean() - t_gas) > 0.02
    assert abs(T1[~near].mean() - t_gas) < 0.01


def _moving_box(nx=6, nyz=2, seed=43):
    mesh = I.box_mesh((nx, nyz, nyz), (1.0, 0.5, 0.5), (False, True, True), jitter=0.1, seed=seed)
    mesh["bkind"] = I.boundary_kinds(mesh, {(0, "lo"): I.BC_NOSLIP_WALL, (0, "hi"): I.BC_MOVING_WALL})
    return mesh


def test_moving_wall_at_rest_is_the_noslip_wall(oracle_mod):
    """A moving wall with zero velocity is the non-slip adiabatic wall: the
    face records agree to rounding."""
    mesh = _moving_box()
    W, dW = _smooth_state(mesh)
    om = oracle_mod.Mesh(mesh)
    mesh2 = dict(mesh)
    mesh2["bkind"] = I.boundary_kinds(mesh, {(0, "lo"): I.BC_NOSLIP_WALL, (0, "hi"): I.BC_NOSLIP_WALL})
    om2 = oracle_mod.Mesh(mesh2)
    p = oracle_mod.params(weno=1, viscous=1, mu=0.01, wall_velocity=(0.0, 0.0, 0.0))
    for stage in (1, 2):
        a = om.face_records(p, W, dW, 2e-3, stage)
        b = om2.face_records(p, W, dW, 2e-3, stage)
        assert np.abs(a - b).max() < 1e-14 * np.abs(b).max()


def test_gas_moving_with_the_wall_stays_uniform(oracle_mod):
    """Gas moving along the walls with the walls' velocity (both x ends
    moving with U_w = (0, 0.3, -0.2)) is a uniform steady flow: the moving
    wall's ghost is then the interior state itself."""
    mesh = I.box_mesh((4, 2, 2), (1.0, 0.5, 0.5), (False, True, True), jitter=0.1, seed=44)
    mesh["bkind"] = I.boundary_kinds(mesh, {(0, "lo"): I.BC_MOVING_WALL, (0, "hi"): I.BC_MOVING_WALL})
    nc = mesh["tet"].shape[0]
    U = np.array([0.0, 0.3, -0.2])
    W = np.zeros((5, nc))
    W[0], W[1:4], W[4] = 1.1, 1.1 * U[:, None], 1.0 / 0.4 + 0.5 * 1.1 * U @ U
    om = oracle_mod.Mesh(mesh)
    p = oracle_mod.params(weno=1, cfl=0.5, viscous=1, mu=0.01, wall_velocity=tuple(U))
    W1, dW1, _, _ = om.run(p, W, np.zeros((15, nc)), nsteps=5)
    assert np.abs(W1 - W).max() < 1e-13
    assert np.abs(dW1).max() < 1e-12


def test_moving_wall_drives_the_gas(oracle_mod):
    """Gas at rest; the x = 1 wall moves along y: the gas next to the moving
    wall picks up y momentum (the viscous shear) while the far side has not
    felt it yet, and the wall does work on the gas.  The ghost is the
    at-rest one in the wall's frame, but the flux is evaluated at a fixed
    point that the wall slides past, so with tangential gradients a little
    mass (here 2e-6 of it in 6 steps) crosses the moving wall."""
    mesh = _moving_box()
    nc = mesh["tet"].shape[0]
    W = np.zeros((5, nc))
    W[0], W[4] = 1.0, 1.0 / 0.4
    om = oracle_mod.Mesh(mesh)
    geo = om.geometry()
    vol, cx = geo["vol"], geo["cen"][:, 0]
    p = oracle_mod.params(weno=1, cfl=0.5, viscous=1, mu=0.02, wall_velocity=(0.0, 0.3, 0.0))
    W1, _, _, _ = om.run(p, W, np.zeros((15, nc)), nsteps=6)
    assert abs((vol * W1[0]).sum() - (vol * W[0]).sum()) < 1e-5 * (vol * W[0]).sum()
    v = W1[2] / W1[0]
    assert v[cx > 5.0 / 6.0].mean() > 0.02
    assert abs(v[cx < 1.0 / 6.0].mean()) < 1e-3
    assert (vol * W1[4]).sum() > (vol * W[4]).sum()
