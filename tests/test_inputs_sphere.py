"""The sphere's O-type shell mesh (inputs.sphere_shell_mesh): cell count with
the pole rows, a closed conforming mesh (every interior face shared by two
tets, so the only boundary faces are the two spheres), positive volumes, the
shell's volume approached under refinement, and the boundary kinds."""
import math

import numpy as np
import pytest

from paper_2102_01366_gb300 import inputs as I


@pytest.mark.parametrize("n", [(3, 6, 12), (2, 7, 10), (4, 8, 16)])
def test_shell_counts_and_closure(oracle_mod, n):
    nr, nt, nphi = n
    m = I.sphere_shell_mesh(nr, nt, nphi, 0.5, 1.5, 1.08)
    nc = m["tet"].shape[0]
    assert nc == 6 * nr * (nt - 2) * nphi + 3 * nr * 2 * nphi
    o = oracle_mod.Mesh(m)
    top = o.topology()
    lr = top["face_lr"]
    nb = int((lr < 0).sum())
    # wall and far-field spheres: two triangles per quad, one per pole triangle
    per_sphere = 2 * (nt - 2) * nphi + 2 * nphi
    assert nb == 2 * per_sphere
    assert (4 * nc - nb) % 2 == 0 and o.nf == (4 * nc - nb) // 2 + nb
    kinds = m["bkind"]
    assert (kinds == I.BC_NOSLIP_WALL).sum() == per_sphere
    assert (kinds == I.BC_FIXED).sum() == per_sphere
    # the kinds sit exactly on the boundary faces
    nbr = top["nbr"]
    assert ((kinds != 0) == (nbr < 0)).all()
    geo = o.geometry()
    assert (geo["vol"] > 0).all()
    r = np.linalg.norm(geo["cen"], axis=1)
    assert r.min() > 0.5 and r.max() < 1.5


def test_shell_volume_converges():
    exact = 4.0 / 3.0 * math.pi * (1.5 ** 3 - 0.5 ** 3)
    errs = []
    for nt, nphi in ((6, 12), (12, 24), (24, 48)):
        m = I.sphere_shell_mesh(2, nt, nphi, 0.5, 1.5, 1.0)
        x = m["xyz"][m["tet"]]
        vol = np.einsum("ij,ij->i", x[:, 1] - x[:, 0], np.cross(x[:, 2] - x[:, 0], x[:, 3] - x[:, 0])) / 6.0
        assert (vol > 0).all()
        errs.append(abs(vol.sum() - exact) / exact)
    # inscribed polyhedra: second order in the angular spacing
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] / errs[2] > 3.5


def test_radial_spacing_is_geometric():
    m = I.sphere_shell_mesh(6, 4, 8, 0.5, 20.0, 1.08)
    north = m["xyz"][:7, 2]  # the north-pole vertex of every radius
    dr = np.diff(north)
    np.testing.assert_allclose(dr[1:] / dr[:-1], 1.08, rtol=1e-12)
    assert north[0] == 0.5 and abs(north[-1] - 20.0) < 1e-12


def test_sphere_case_free_stream():
    m, W, dW, mu = I.sphere_case(2, 6, 8)
    assert W.shape == (5, m["tet"].shape[0]) and not dW.any()
    np.testing.assert_allclose(W[:, 0], [1.0, 0.2, 0.0, 0.0, (1 / 1.4) / 0.4 + 0.02])
    assert abs(mu - 0.2 * 1.0 / 100.0) < 1e-15
