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
