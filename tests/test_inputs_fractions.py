"""The input generator's exact volume fractions (the Riemann-slab initial
states of the batched workload), against closed forms; no GPU."""
import numpy as np
import pytest

from paper_2102_01366_gb300 import inputs as I


@pytest.mark.parametrize("t", [0.1, 0.37, 0.5, 0.9])
def test_fraction_below_a_plane_in_a_corner_tetrahedron(t):
    """Vertices at x = 0, 0, 0, 1: the part with x < t has volume fraction
    1 - (1 - t)^3 (the cut-off apex is similar with ratio 1 - t); three
    equal vertex values exercise the separation of ties."""
    d = np.array([[-t, -t, -t, 1.0 - t]])
    assert abs(I._neg_fraction(d)[0] - (1.0 - (1.0 - t) ** 3)) < 1e-7


def test_fraction_is_zero_or_one_off_the_plane_and_complements():
    rng = np.random.Generator(np.random.PCG64(4))
    d = rng.standard_normal((2000, 4))
    f = I._neg_fraction(d)
    g = I._neg_fraction(-d)
    assert np.all((f >= 0) & (f <= 1))
    np.testing.assert_allclose(f + g, 1.0, atol=1e-7)
    assert np.all(f[(d > 0).all(1)] == 0.0) and np.all(f[(d < 0).all(1)] == 1.0)


def test_slab_volume_on_the_jittered_periodic_cube():
    """The slab 0.25 <= x < 0.75 of the periodic unit cube has volume 0.5;
    the cells' fractions inside it, weighted by their volumes (from the
    vertex determinants), must add up to that, and the slab state's
    density must carry the matching mass."""
    mesh = I.box_mesh((9, 9, 9), jitter=0.1, seed=11, diagonal=(1, 1, -1))
    v = I.tet_vertices(mesh)
    vol = np.abs(np.linalg.det(v[:, 1:] - v[:, :1])) / 6.0
    assert abs(vol.sum() - 1.0) < 1e-12
    x = v[:, :, 0]
    frac = I._neg_fraction(x - 0.75) - I._neg_fraction(x - 0.25)
    assert abs(frac @ vol - 0.5) < 1e-8
    W, _ = I.riemann_slab_state(mesh, inner=(1.0, 1.0), outer=(0.125, 0.1), mach=1.0)
    assert abs(W[0] @ vol - (0.5 * 1.0 + 0.5 * 0.125)) < 1e-8


def _dirichlet_mean(X, expo):
    """Mean over the tetrahedron with vertices X [4, 3] of prod_d x_d^expo[d]:
    x = sum_v lam_v X_v with lam uniform on the simplex (Dirichlet(1,1,1,1)),
    E[prod_v lam_v^k_v] = 3! prod_v k_v! / (3 + sum_v k_v)!."""
    import itertools
    import math
    factors = [d for d in range(3) for _ in range(expo[d])]
    tot = 0.0
    for idx in itertools.product(range(4), repeat=len(factors)):
        k = np.bincount(np.array(idx, dtype=int), minlength=4)
        e = 6.0 * np.prod([math.factorial(int(a)) for a in k]) / math.factorial(3 + len(factors))
        tot += e * np.prod([X[i, d] for i, d in zip(idx, factors)])
    return tot


@pytest.mark.parametrize("order", [2, 3, 5])
def test_cell_average_rule_is_exact_to_degree_2n_minus_3(order):
    """The collapsed Gauss-Legendre rule behind every initial cell average
    (n points per direction on the Duffy map, whose Jacobian adds degree 2)
    integrates polynomials of total degree <= 2n - 3 exactly."""
    import itertools
    rng = np.random.Generator(np.random.PCG64(order))
    X = rng.standard_normal((3, 4, 3))
    mesh = {"xyz": X.reshape(12, 3), "tet": np.arange(12).reshape(3, 4),
            "shift": np.zeros((3, 4, 3), np.int8), "period": np.zeros(3)}
    expos = [e for e in itertools.product(range(2 * order - 2), repeat=3) if sum(e) <= 2 * order - 3]
    f = lambda x: np.stack([x[..., 0] ** e[0] * x[..., 1] ** e[1] * x[..., 2] ** e[2] for e in expos], -1)
    got = I.cell_average(mesh, f, order=order)
    for c in range(3 if order < 5 else 1):  # the closed form costs 4^degree terms
        ref = np.array([_dirichlet_mean(X[c], e) for e in expos])
        np.testing.assert_allclose(got[c], ref, rtol=1e-12, atol=1e-12)
