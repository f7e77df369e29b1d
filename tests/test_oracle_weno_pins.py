"""Exact pins of the oracle's WENO pieces (Sec. 4.2 and Sec. 4.3) against
values that do not come from the oracle's own formulas:

* the smoothness indicators of Eq. smooth-indicator for random linear and
  quadratic polynomials on jittered tetrahedra, against the closed-form
  integral of an affine function squared over a tetrahedron,
  int_T (sum_k lambda_k d_k)^2 = |T| / 20 (sum_k d_k^2 + (sum_k d_k)^2),
  applied to each first derivative (affine in x) with d_k its vertex values;
* beta_0 of the two-step reconstruction (Eq. p0-non-linear-weight) and the
  nonlinear weights (Eq. non-linear-weight), against hand-worked exact
  fractions in tests/golden/weno_weights.txt;
* the combination of Eq. final_weno_expression-3rd, through what it implies
  for R: its quadratic part is wbar_2 / gamma_2,2 times that of P^2, and its
  linear part follows from P^2's and P^1's with the weights.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2102_01366_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden", "weno_weights.txt")
PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def _frac(s):
    return float(Fraction(s))


def _golden():
    beta0, weights = [], []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, *rest = [p.strip() for p in line.split("|")]
        kind, name, *nums = head.split()
        if kind == "beta0":
            vol, eps = float(nums[0]), float(nums[1])
            b = [[float(x) for x in row.split()] for row in rest[0].split(";")]
            beta0.append((name, vol, eps, np.array(b), _frac(rest[1]), [_frac(x) for x in rest[2].split()],
                          _frac(rest[3])))
        else:
            order, eps, b0, b1, b2 = int(nums[0]), float(nums[1]), float(nums[2]), float(nums[3]), float(nums[4])
            weights.append((name, order, eps, b0, b1, b2, [_frac(x) for x in rest[0].split()]))
    return beta0, weights


BETA0, WEIGHTS = _golden()


def _affine_square_integral(vol, d):
    """int over a tet of an affine function with vertex values d[4], squared."""
    return vol / 20.0 * ((d * d).sum() + d.sum() ** 2)


def _grad_at(v, X):
    """gradient of the basis-form polynomial v[10] at X (relative to the
    centroid): the linear part v[1..3] plus the derivative of the quadratic
    monomials X_i X_j (the basis means do not depend on X)."""
    g = np.array(v[1:4], dtype=np.float64)
    for q, (i, j) in enumerate(PAIRS):
        g[i] += v[4 + q] * X[j]
        g[j] += v[4 + q] * X[i]
    return g


def _beta_closed_form(verts, v, r):
    e = verts[1:] - verts[0]
    vol = abs(np.linalg.det(e)) / 6.0
    cen = verts.mean(0)
    grads = np.array([_grad_at(v, x - cen) for x in verts])  # [4 vertices][3]
    first = sum(_affine_square_integral(vol, grads[:, l]) for l in range(3))
    beta = vol ** (2.0 / 3.0 - 1.0) * first
    if r == 2:
        # the six distinct second derivatives: d2/dx_i^2 of X_i^2 is 2
        dd = [(2.0 if i == j else 1.0) * v[4 + q] for q, (i, j) in enumerate(PAIRS)]
        beta += vol ** (4.0 / 3.0 - 1.0) * vol * sum(x * x for x in dd)
    return beta


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_smoothness_indicator_closed_form(oracle_mod, seed):
    mesh = I.box_mesh((2, 2, 2), jitter=0.1, seed=60 + seed)
    om = oracle_mod.Mesh(mesh)
    verts = I.tet_vertices(mesh)
    rng = np.random.default_rng(seed)
    for c in rng.choice(om.nc, 6, replace=False):
        # linear P (r = 1): beta_1 = |Omega|^(2/3) |b|^2 exactly
        v1 = np.zeros(10)
        v1[0], v1[1:4] = rng.normal(), rng.normal(size=3)
        b1 = om.smoothness(c, v1, 1)
        assert b1 == pytest.approx(_beta_closed_form(verts[c], v1, 1), rel=1e-13)
        vol = abs(np.linalg.det(verts[c][1:] - verts[c][0])) / 6.0
        assert b1 == pytest.approx(vol ** (2.0 / 3.0) * (v1[1:4] ** 2).sum(), rel=1e-13)
        # quadratic P (r = 2); curvature large enough that both terms count
        v2 = np.zeros(10)
        v2[0], v2[1:4], v2[4:] = rng.normal(), rng.normal(size=3), 10.0 * rng.normal(size=6)
        want = _beta_closed_form(verts[c], v2, 2)
        got = om.smoothness(c, v2, 2)
        assert got == pytest.approx(want, rel=1e-12), (c, got, want)
        # both parts are material: each is > 1 % of the indicator
        second = vol ** (4.0 / 3.0) * sum(((2.0 if i == j else 1.0) * v2[4 + q]) ** 2 for q, (i, j) in enumerate(PAIRS))
        assert 0.01 < second / want < 0.99


@pytest.mark.parametrize("case", BETA0, ids=[c[0] for c in BETA0])
def test_two_step_beta0_hand_values(oracle_mod, case):
    name, vol, eps, b, sigma1, wbar1, beta0 = case
    got, s1, w1 = oracle_mod.weno_beta0(vol, b, eps=eps)
    assert s1 == pytest.approx(sigma1, rel=1e-14, abs=1e-300)
    np.testing.assert_allclose(w1, wbar1, rtol=1e-14)
    assert got == pytest.approx(beta0, rel=1e-14)


@pytest.mark.parametrize("case", WEIGHTS, ids=[c[0] for c in WEIGHTS])
def test_nonlinear_weights_hand_values(oracle_mod, case):
    name, order, eps, b0, b1, b2, wbar = case
    got = oracle_mod.weno_weights(order, b0, b1, b2, eps=eps)
    np.testing.assert_allclose(got, wbar, rtol=1e-14, atol=1e-300)


def test_weights_tend_to_linear_weights_when_smooth(oracle_mod):
    """sigma = 0 (equal indicators) leaves the linear weights gamma."""
    np.testing.assert_allclose(oracle_mod.weno_weights(3, 0.3, 0.3, 0.3), [1 / 111, 10 / 111, 100 / 111], rtol=1e-15)
    np.testing.assert_allclose(oracle_mod.weno_weights(2, 0.3, 0.3), [1 / 11, 10 / 11, 0.0], rtol=1e-15)


def test_reconstruction_combines_the_weighted_polynomials(oracle_mod):
    """Eq. final_weno_expression-3rd with p_1 = (P^1 - g01 P^0)/g11 and
    p_2 = (P^2 - g12 p_1 - g02 p_0)/g22: R's second derivatives are
    wbar_2/g22 times P^2's, and its first derivatives at the centroid are
    wbar_2/g22 grad P^2 + (wbar_1 - wbar_2 g12/g22)/g11 grad P^1, the
    weights taken from the pinned pieces above with the indicators of the
    cell's own P^1, P^2 and its neighbours' step-1 slopes.  Checked on the
    cells of a Sod tube next to the jump, where the weights are far from
    linear."""
    mesh = I.box_mesh((12, 2, 2), (1.0, 1 / 6, 1 / 6), (False, True, True), jitter=0.1, seed=34)
    W, dW = I.riemann_x_state(mesh)
    om = oracle_mod.Mesh(mesh)
    p_weno = oracle_mod.params(weno=1)
    R, b, fb = om.reconstruct(p_weno, W, dW)
    P2, _, fb2 = om.reconstruct(oracle_mod.params(weno=0), W, dW)
    geo, topo = om.geometry(), om.topology()
    g22, g12, g11 = 100 / 111, 10 / 111, 10 / 11
    checked = 0
    far = 0
    for c in range(om.nc):
        nb = topo["nbr"][c]
        if (nb < 0).any() or fb[c] or fb2[c]:
            continue  # boundary cells (one-sided stencil); cells whose R or P^2 fell back
        vol = geo["vol"][c]
        for q in range(5):
            # basis form of P^1 and P^2 (the quadratic basis has zero mean)
            v1 = np.zeros(10)
            v1[0], v1[1:4] = W[q, c], b[c, q]
            v2 = np.zeros(10)
            v2[0], v2[1:] = W[q, c], P2[c, q, 1:]
            beta1 = om.smoothness(c, v1, 1)
            beta2 = om.smoothness(c, v2, 2)
            beta0, _, _ = oracle_mod.weno_beta0(vol, b[nb, q], eps=p_weno.eps_weno)
            w = oracle_mod.weno_weights(3, beta0, beta1, beta2, eps=p_weno.eps_weno)
            a2 = w[2] / g22
            a1 = (w[1] - w[2] * g12 / g22) / g11
            scale = np.abs(P2[c, q, 1:]).max() + np.abs(b[c, q]).max() + 1e-300
            np.testing.assert_allclose(R[c, q, 4:], a2 * P2[c, q, 4:], rtol=0, atol=1e-13 * scale)
            np.testing.assert_allclose(R[c, q, 1:4], a2 * P2[c, q, 1:4] + a1 * b[c, q], rtol=0, atol=1e-13 * scale)
            checked += 1
            far += abs(w[2] - g22) > 0.1
    assert checked > 100 and far > 10
