"""The oracle's constrained reconstruction at non-slip adiabatic walls
(Sec. 4.4), pinned by what the definition fixes:

* the constraint: for any data, a wall cell's momentum P1 vanishes at the
  centroid of each wall face and its P2 at the face's three Gauss points
  (the wall velocity is zero);
* exactness: a momentum field in the constrained space (linear or
  quadratic, zero on the wall) is reproduced exactly by the constrained
  least squares, since it fits every datum with zero residual;
* locality: density and energy, and every cell without a wall face, are
  reconstructed as without the constraint;
* with the constraint off nothing vanishes at the wall (the pins can fail).
"""
import numpy as np
import pytest

from paper_2102_01366_gb300 import inputs as I


def _wall_box(nx=3, seed=71, hi=I.BC_OPEN):
    # no periodic axis, so that any polynomial field gives consistent data
    mesh = I.box_mesh((nx, 3, 3), (1.0, 1.0, 1.0), (False, False, False), jitter=0.1, seed=seed)
    mesh["bkind"] = I.boundary_kinds(mesh, {(0, "lo"): I.BC_NOSLIP_WALL, (0, "hi"): hi})
    return mesh


def _mono(P, X):
    """R in centroid-monomial form (c0, x, y, z, xx, xy, xz, yy, yz, zz) at offsets X[..., 3]."""
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    return (P[0] + P[1] * x + P[2] * y + P[3] * z + P[4] * x * x + P[5] * x * y + P[6] * x * z +
            P[7] * y * y + P[8] * y * z + P[9] * z * z)


def _wall_points(om, mesh):
    """For each cell: its wall faces' Gauss points relative to its centroid [k][3][3]."""
    top, geo = om.topology(), om.geometry()
    out = {}
    for c in range(om.nc):
        pts = []
        for f in range(4):
            if top["nbr"][c, f] >= 0 or mesh["bkind"][c, f] != I.BC_NOSLIP_WALL:
                continue
            fi = top["csr_face"][c, f]
            gp = geo["gp_l"][fi] if top["csr_sign"][c, f] > 0 else geo["gp_r"][fi]
            pts.append(gp.reshape(3, 3))
        if pts:
            out[c] = np.array(pts)
    return out


def _random_state(nc, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    W = np.empty((5, nc))
    W[0] = 1.0 + 0.2 * rng.random(nc)
    W[1:4] = 0.1 * rng.standard_normal((3, nc))
    W[4] = 5.0 + rng.random(nc)
    dW = 0.1 * rng.standard_normal((15, nc))
    return W, dW


def test_wall_cells_get_constrained_stencils(oracle_mod):
    mesh = _wall_box()
    om = oracle_mod.Mesh(mesh)
    pts = _wall_points(om, mesh)
    MW1, MW2, wc = om.wall_stencils()
    assert set(np.nonzero(wc)[0]) == set(pts)  # every wall cell, and only those
    assert len(pts) == 18  # 3 x 3 hexahedra on the wall, 2 tetrahedra each
    # without wall faces nothing is built
    mesh0 = dict(mesh, bkind=I.boundary_kinds(mesh, {}))
    assert oracle_mod.Mesh(mesh0).wall_stencils()[2].sum() == 0


@pytest.mark.parametrize("order", [2, 3])
def test_momentum_vanishes_at_the_wall_for_any_data(oracle_mod, order):
    """Linear weights: R = P1 (order 2) vanishes at each wall face's
    centroid, R = P2 (order 3) at its three Gauss points."""
    mesh = _wall_box()
    om = oracle_mod.Mesh(mesh)
    pts = _wall_points(om, mesh)
    W, dW = _random_state(om.nc, 5)
    poly, _, fb = om.reconstruct(oracle_mod.params(weno=0, order=order, wall_constraint=1), W, dW)
    poly0, _, _ = om.reconstruct(oracle_mod.params(weno=0, order=order, wall_constraint=0), W, dW)
    scale = np.abs(W[1:4]).max()
    worst, worst0 = 0.0, 0.0
    for c, P in pts.items():
        assert not fb[c]
        X = P.mean(axis=1) if order == 2 else P.reshape(-1, 3)
        for q in (1, 2, 3):
            worst = max(worst, np.abs(_mono(poly[c, q], X)).max())
            worst0 = max(worst0, np.abs(_mono(poly0[c, q], X)).max())
    assert worst < 1e-13 * scale, worst
    assert worst0 > 1e-2 * scale  # unconstrained: no reason to vanish there


@pytest.mark.parametrize("weno", [0, 1])
def test_slopes_vanish_at_wall_face_centroids(oracle_mod, weno):
    """Step 1 (the slopes every weight choice uses): Q0 + b.(x_f - x_c) = 0
    at each wall face's centroid."""
    mesh = _wall_box(seed=72)
    om = oracle_mod.Mesh(mesh)
    pts = _wall_points(om, mesh)
    W, dW = _random_state(om.nc, 6)
    _, slopes, _ = om.reconstruct(oracle_mod.params(weno=weno, wall_constraint=1), W, dW)
    for c, P in pts.items():
        for xf in P.mean(axis=1):
            for q in (1, 2, 3):
                assert abs(W[q, c] + slopes[c, q] @ xf) < 1e-13 * np.abs(W[1:4]).max()


def _field(coef):
    """Momentum fields zero on the wall x = 0: rho U_q = x (a + b x + c y + d z)."""
    def f(x):
        out = np.empty(x.shape[:-1] + (5,))
        out[..., 0] = 1.0 + 0.1 * x[..., 1]
        for q in (1, 2, 3):
            a, b, c, d = coef[q - 1]
            out[..., q] = x[..., 0] * (a + b * x[..., 0] + c * x[..., 1] + d * x[..., 2])
        out[..., 4] = 2.5 + 0.2 * x[..., 2]
        return out
    return f


def _averages(mesh, f, h=1e-5):
    """Cell averages of f and of its gradient (central differences of the
    averages of shifted fields: exact for these quadratics up to rounding)."""
    W = I.cell_average(mesh, f).T
    dW = np.zeros((15, W.shape[1]))
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        Wp = I.cell_average(mesh, lambda x: f(x + e)).T
        Wm = I.cell_average(mesh, lambda x: f(x - e)).T
        for q in range(5):
            dW[3 * q + i] = (Wp[q] - Wm[q]) / (2 * h)
    return W, dW


@pytest.mark.parametrize("order,linear", [(3, False), (2, True)])
def test_fields_zero_on_the_wall_are_reproduced(oracle_mod, order, linear):
    """A quadratic (order 3) or linear (order 2) momentum field that is zero
    on the wall satisfies every constraint and fits all stencil data with
    zero residual, so the constrained fit returns it: R equals the field at
    every Gauss point of the wall cell's faces."""
    rng = np.random.Generator(np.random.PCG64(9))
    coef = rng.standard_normal((3, 4))
    if linear:
        coef[:, 1:] = 0.0
    mesh = _wall_box(seed=73)
    om = oracle_mod.Mesh(mesh)
    pts = _wall_points(om, mesh)
    f = _field(coef)
    W, dW = _averages(mesh, f)
    poly, _, _ = om.reconstruct(oracle_mod.params(weno=0, order=order, wall_constraint=1), W, dW)
    geo, top = om.geometry(), om.topology()
    cen = geo["cen"]
    worst = 0.0
    for c in pts:
        X = []
        for f4 in range(4):
            fi = top["csr_face"][c, f4]
            gp = geo["gp_l"][fi] if top["csr_sign"][c, f4] > 0 else geo["gp_r"][fi]
            X.append(gp.reshape(3, 3))
        X = np.concatenate(X)
        exact = f(cen[c] + X)
        for q in (1, 2, 3):
            worst = max(worst, np.abs(_mono(poly[c, q], X) - exact[:, q]).max())
    assert worst < 1e-8, worst  # the gradient data carry the 1e-10 central-difference error


def test_density_energy_and_other_cells_are_unchanged(oracle_mod):
    mesh = _wall_box(seed=74)
    om = oracle_mod.Mesh(mesh)
    _, _, wc = om.wall_stencils()
    W, dW = _random_state(om.nc, 7)
    for weno in (0, 1):
        a, sa, _ = om.reconstruct(oracle_mod.params(weno=weno, wall_constraint=1), W, dW)
        b, sb, _ = om.reconstruct(oracle_mod.params(weno=weno, wall_constraint=0), W, dW)
        np.testing.assert_array_equal(a[:, [0, 4]], b[:, [0, 4]])
        np.testing.assert_array_equal(sa[:, [0, 4]], sb[:, [0, 4]])
        if weno == 0:
            # linear weights: a cell's R reads only its own stencil
            np.testing.assert_array_equal(a[wc == 0], b[wc == 0])
        else:
            # WENO: a wall cell's neighbours read its (constrained) slopes in
            # their two-step beta_0; the rest are untouched
            top = om.topology()
            near = wc.astype(bool).copy()
            for c in np.nonzero(wc)[0]:
                near[top["nbr"][c][top["nbr"][c] >= 0]] = True
            np.testing.assert_array_equal(a[~near], b[~near])


def test_closed_box_with_constrained_walls_conserves_mass_and_energy(oracle_mod):
    mesh = _wall_box(nx=4, seed=75, hi=I.BC_NOSLIP_WALL)
    mesh["bkind"] = I.boundary_kinds(mesh, {(a, e): I.BC_NOSLIP_WALL for a in range(3) for e in ("lo", "hi")})
    om = oracle_mod.Mesh(mesh)
    vol = om.geometry()["vol"]
    x = om.geometry()["cen"]
    nc = om.nc
    W = np.zeros((5, nc))
    W[0] = 1.0 + 0.1 * np.sin(3 * x[:, 0])
    W[1] = 0.2 * np.sin(np.pi * x[:, 0]) * W[0]
    W[4] = 2.5 + 0.5 * (W[1] ** 2) / W[0]
    dW = np.zeros((15, nc))
    W1, _, _, _ = om.run(oracle_mod.params(weno=1, cfl=0.5, viscous=1, mu=0.01, wall_constraint=1), W, dW,
                         nsteps=4)
    tot0, tot1 = (W * vol).sum(1), (W1 * vol).sum(1)
    for q in (0, 4):
        assert abs(tot1[q] - tot0[q]) < 1e-14 * abs(tot0[q]), q
