"""Pins of the oracle's mesh topology, geometry and quadrature (Sec. 2.1,
Sec. 4.1) against closed forms that do not use the oracle's own formulas."""
import math

import numpy as np
import pytest

from paper_2102_01366_gb300 import inputs as I


def _mesh(n=(3, 3, 3), periodic=(True, True, True), length=(1.0, 1.0, 1.0), seed=5):
    return I.box_mesh(n, length, periodic, jitter=0.1, seed=seed)


def _simplex_integral(exps):
    """int over a tet of prod_k lambda_k^a_k = 6|T| a0!a1!a2!a3!/(sum a + 3)!,
    returned per unit 6|T|."""
    num = 1.0
    for a in exps:
        num *= math.factorial(a)
    return num / math.factorial(sum(exps) + 3)


@pytest.mark.parametrize("periodic", [(True, True, True), (False, True, True)])
def test_volume_centroid_moments_closed_form(oracle_mod, periodic):
    mesh = _mesh(periodic=periodic)
    om = oracle_mod.Mesh(mesh)
    g = om.geometry()
    v = I.tet_vertices(mesh)
    vol = np.einsum("ci,ci->c", np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), v[:, 3] - v[:, 0]) / 6.0
    np.testing.assert_allclose(g["vol"], vol, rtol=1e-13)
    assert abs(g["vol"].sum() - 1.0) < 1e-13  # the tets tile the unit box
    # centroid and second moments from the simplex monomial integrals:
    # x = sum_k lambda_k v_k, so int x_i x_j = sum_kl v_ki v_lj int lambda_k lambda_l
    cen = v.mean(1)
    np.testing.assert_allclose(g["cen"], cen, rtol=0, atol=1e-15)
    Ikl = np.empty((4, 4))
    for k in range(4):
        for l in range(4):
            e = [0, 0, 0, 0]
            e[k] += 1
            e[l] += 1
            Ikl[k, l] = _simplex_integral(e) * 6.0  # per unit volume
    y = v - cen[:, None, :]
    M = np.einsum("kl,cki,clj->cij", Ikl, y, y)
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for q, (i, j) in enumerate(pairs):
        np.testing.assert_allclose(g["mom2"][:, q], M[:, i, j], rtol=1e-12, atol=1e-18)


@pytest.mark.parametrize("periodic", [(True, True, True), (False, True, True)])
def test_topology_consistency(oracle_mod, periodic):
    mesh = _mesh(periodic=periodic)
    om = oracle_mod.Mesh(mesh)
    t = om.topology()
    nc, nf = om.nc, om.nf
    # every cell has 4 distinct faces; every face appears once per side
    assert all(len(set(r)) == 4 for r in t["csr_face"])
    seen = np.zeros((nf, 2), np.int64)
    for c in range(nc):
        for f in range(4):
            fi = t["csr_face"][c, f]
            side = 0 if t["csr_sign"][c, f] > 0 else 1
            assert t["face_lr"][fi, side] == c
            seen[fi, side] += 1
            nb = t["nbr"][c, f]
            other = t["face_lr"][fi, 1 - side]
            assert nb == other
            if nb >= 0:
                assert c in t["nbr"][nb]
    assert ((seen == 1) | (t["face_lr"] == -1)).all()
    # faces sorted lexicographically by their sorted vertex ids
    fv = t["face_v"]
    assert (np.diff(fv, axis=1) > 0).all()
    keys = [tuple(r) for r in fv]
    assert keys == sorted(keys)
    if all(periodic):
        assert nf == 2 * nc and (t["face_lr"] >= 0).all()
    else:
        nb = (t["face_lr"] < 0).any(1).sum()
        assert nb == 2 * 2 * mesh["n"][1] * mesh["n"][2]  # two triangles per hex side, two ends


def test_face_orientation_and_closure(oracle_mod):
    mesh = _mesh(periodic=(False, True, True))
    om = oracle_mod.Mesh(mesh)
    g, t = om.geometry(), om.topology()
    n = g["fnorm"]
    # canonical sign: first nonzero component positive; unit length
    first = np.where(n[:, 0] != 0, n[:, 0], np.where(n[:, 1] != 0, n[:, 1], n[:, 2]))
    assert (first > 0).all()
    np.testing.assert_allclose(np.linalg.norm(n, axis=1), 1.0, rtol=1e-14)
    # left cell: the normal points out of it (from its centroid to the face)
    for f in range(om.nf):
        l, r = t["face_lr"][f]
        if l >= 0:
            assert np.dot(g["gp_l"][f].mean(0), n[f]) > 0
        if r >= 0:
            assert np.dot(g["gp_r"][f].mean(0), n[f]) < 0
    # closed surface: sum over the cell's faces of s * A * n = 0
    S = np.zeros((om.nc, 3))
    for c in range(om.nc):
        for f in range(4):
            fi = t["csr_face"][c, f]
            S[c] += t["csr_sign"][c, f] * g["farea"][fi] * n[fi]
    assert np.abs(S).max() < 1e-15
    # inscribed-radius estimate 3|Omega| / sum |Gamma|
    A = np.array([g["farea"][t["csr_face"][c]].sum() for c in range(om.nc)])
    np.testing.assert_allclose(g["dr"], 3 * g["vol"] / A, rtol=1e-14)


def test_face_rule_exact_for_quadratics(oracle_mod):
    """3-point rule with weights A/3 integrates quadratics over each face
    exactly (Sec. 2.1); the exact value comes from barycentric monomial
    integrals int lambda^a = 2A a!b!c!/(a+b+c+2)!."""
    mesh = _mesh()
    om = oracle_mod.Mesh(mesh)
    g, t = om.geometry(), om.topology()
    rng = np.random.default_rng(0)
    c0, c1, H = rng.normal(), rng.normal(size=3), rng.normal(size=(3, 3))
    H = H + H.T
    for f in range(0, om.nf, 7):
        L = t["face_lr"][f, 0]
        x = g["gp_l"][f] + g["cen"][L]  # absolute, left frame
        q = lambda y: c0 + y @ c1 + 0.5 * y @ H @ y
        approx = g["farea"][f] / 3.0 * sum(q(x[k]) for k in range(3))
        # vertices of the face (left frame) from its Gauss points:
        # x_k = v_k / 2 + (v_0 + v_1 + v_2) / 6
        Bm = np.full((3, 3), 1.0 / 6.0) + 0.5 * np.eye(3)
        V = np.linalg.solve(Bm, x)
        A = g["farea"][f]
        # polynomial in barycentric coordinates: q(sum l_k V_k)
        exact = c0 * A
        exact += (V.mean(0) @ c1) * A
        Iab = np.array([[2 * A * (2 if a == b else 1) / math.factorial(4) for b in range(3)] for a in range(3)])
        exact += 0.5 * np.einsum("ab,ai,bj,ij->", Iab, V, V, H)
        assert abs(approx - exact) < 1e-14 * max(1.0, abs(exact))


def test_rejects_bad_meshes(oracle_mod):
    mesh = _mesh()
    bad = dict(mesh)
    tet = mesh["tet"].copy()
    tet[0, [1, 2]] = tet[0, [2, 1]]  # negative orientation
    bad["tet"] = tet
    with pytest.raises(ValueError):
        oracle_mod.Mesh(bad)
    dup = dict(mesh)
    dup["tet"] = np.concatenate([mesh["tet"], mesh["tet"][:1]])
    dup["shift"] = np.concatenate([mesh["shift"], mesh["shift"][:1]])
    with pytest.raises(ValueError):
        oracle_mod.Mesh(dup)
