"""The C-ABI library on the host (no GPU): every declared entry point is
exported, and the host mesh setup reproduces the oracle's connectivity bit
for bit, its FP64 geometry and its least-squares operators to rounding."""
import ctypes as C

import numpy as np
import pytest

from paper_2102_01366_gb300 import gks
from paper_2102_01366_gb300 import inputs as I

MESHES = {
    "periodic2": lambda: I.box_mesh((2, 2, 2), jitter=0.1, seed=1),
    "periodic3_diag": lambda: I.box_mesh((3, 3, 4), jitter=0.1, seed=2, diagonal=(1, 1, -1)),
    "sod_like": lambda: I.box_mesh((6, 2, 3), (1.0, 0.2, 0.3), (False, True, True), jitter=0.1, seed=3),
    "uniform": lambda: I.box_mesh((3, 3, 3), jitter=0.0, seed=0),
    "open_z": lambda: I.box_mesh((3, 3, 3), periodic=(True, True, False), jitter=0.1, seed=4),
}


@pytest.fixture(scope="module")
def built():
    from paper_2102_01366_gb300 import _build
    _build.build()
    return gks.lib()


def test_every_declared_symbol_is_exported(built):
    names = gks.header_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(built, n)]
    assert not missing, missing


@pytest.mark.parametrize("name", sorted(MESHES))
def test_connectivity_bit_exact(built, oracle_mod, name):
    mesh = MESHES[name]()
    g = gks.Mesh(mesh)
    o = oracle_mod.Mesh(mesh)
    assert (g.nc, g.nf) == (o.nc, o.nf)
    tg, to = g.topology(), o.topology()
    for k in ("face_v", "face_lr", "nbr", "csr_face", "csr_sign"):
        np.testing.assert_array_equal(tg[k], to[k], err_msg=k)


@pytest.mark.parametrize("name", sorted(MESHES))
def test_geometry_matches_oracle(built, oracle_mod, name):
    mesh = MESHES[name]()
    gg, go = gks.Mesh(mesh).geometry(), oracle_mod.Mesh(mesh).geometry()
    for k in gg:
        scale = max(np.abs(go[k]).max(), 1e-300)
        assert np.abs(gg[k] - go[k]).max() <= 1e-13 * scale, k
    # the normals are fixed bit for bit by the orientation rule
    assert (np.sign(gg["fnorm"]) == np.sign(go["fnorm"])).all()


@pytest.mark.parametrize("name", sorted(MESHES))
def test_stencils_match_oracle(built, oracle_mod, name):
    mesh = MESHES[name]()
    g = gks.Mesh(mesh)
    o = oracle_mod.Mesh(mesh)
    assert g.n_singular == o.n_singular
    M1g, M2g = g.stencils()
    M1o, M2o = o.stencils()
    # rows scale with powers of h: compare per row relative to the row size
    for Mg, Mo in ((M1g, M1o), (M2g, M2o)):
        scale = np.abs(Mo).max(axis=2, keepdims=True) + 1e-300
        assert (np.abs(Mg - Mo) / scale).max() < 1e-10


WALL_MESHES = {
    # one wall plane; cells on the wall have 3 neighbours and 1 wall face
    "wall_x": lambda: dict(I.box_mesh((3, 3, 3), periodic=(False, True, True), jitter=0.1, seed=6),
                           bkind=None),
    # walls on every face of a closed box: edge and corner cells with 2
    # neighbours and 2 wall faces
    "closed": lambda: dict(I.box_mesh((3, 3, 3), periodic=(False, False, False), jitter=0.1, seed=7),
                           bkind=None),
}


@pytest.mark.parametrize("name", sorted(WALL_MESHES))
def test_wall_stencils_match_oracle(built, oracle_mod, name):
    """The Sec. 4.4 constrained operators of the library (QR null-space
    method) against the oracle's (Gaussian elimination of the KKT system):
    the same cells built, the same operators to rounding."""
    mesh = WALL_MESHES[name]()
    axes = [a for a in range(3) if not mesh["period"][..., a].any()]
    mesh["bkind"] = I.boundary_kinds(mesh, {(a, e): I.BC_NOSLIP_WALL for a in axes for e in ("lo", "hi")})
    g = gks.Mesh(mesh)
    o = oracle_mod.Mesh(mesh)
    W1g, W2g, bg = g.wall_stencils()
    W1o, W2o, bo = o.wall_stencils()
    np.testing.assert_array_equal(bg, bo)
    assert bg.sum() > 0
    for Mg, Mo in ((W1g, W1o), (W2g, W2o)):
        scale = np.abs(Mo).max(axis=2, keepdims=True) + 1e-300
        assert (np.abs(Mg - Mo) / scale).max() < 1e-10
    if name == "closed":
        top = o.topology()
        assert ((top["nbr"] < 0).sum(axis=1)[bg == 1] == 2).any()  # two wall faces


def test_workspace_grows_only_for_constrained_walls(built):
    """wall_constraint = 1 adds one slot of constrained operators per cell
    with a non-slip wall face (168 operator words) plus a slot index per
    cell, and nothing on a mesh without such faces."""
    mesh = I.box_mesh((3, 2, 2), periodic=(False, True, True), jitter=0.1, seed=8)
    plain = gks.Mesh(mesh)
    walled_mesh = dict(mesh, bkind=I.boundary_kinds(mesh, {(0, "lo"): I.BC_NOSLIP_WALL}))
    walled = gks.Mesh(walled_mesh)
    nwall = int(walled.wall_stencils()[2].sum())
    assert nwall == 8
    for prec, word in ((0, 8), (1, 4), (2, 8)):
        def nbytes(g, wc):
            p = gks.params(precision=prec, wall_constraint=wc)
            return gks.lib().gks_workspace_bytes(g._h, C.byref(p))
        assert nbytes(plain, 1) == nbytes(plain, 0)
        extra = nbytes(walled, 1) - nbytes(walled, 0)
        assert extra >= 168 * word * nwall + 4 * plain.nc
        assert extra < 168 * word * nwall + 4 * plain.nc + 512  # two 256-byte alignments
    p = gks.params(wall_constraint=2)
    assert gks.lib().gks_workspace_bytes(walled._h, C.byref(p)) == 0  # invalid option


def test_rejects_bad_input(built):
    mesh = I.box_mesh((3, 3, 3), jitter=0.1, seed=5)
    bad = dict(mesh)
    tet = mesh["tet"].copy()
    tet[3, [1, 2]] = tet[3, [2, 1]]
    bad["tet"] = tet
    with pytest.raises(gks.GksError) as e:
        gks.Mesh(bad)
    assert e.value.status == -2
    bad = dict(mesh)
    tet = mesh["tet"].copy()
    tet[0, 0] = 10 ** 9
    bad["tet"] = tet
    with pytest.raises(gks.GksError) as e:
        gks.Mesh(bad)
    assert e.value.status == -2
    # state creation without a workspace fails before any device call
    g = gks.Mesh(mesh)
    p = gks.params()
    assert gks.lib().gks_workspace_bytes(g._h, C.byref(p)) > 0
    h = C.c_void_p()
    st = gks.lib().gks_state_create(g._h, C.byref(p), None, 0, None, C.byref(h))
    assert st == -7 and not h.value
    p.order = 4
    assert gks.lib().gks_workspace_bytes(g._h, C.byref(p)) == 0
    for field, value in (("prandtl", 0.0), ("wall_temperature", -1.0), ("gamma", 1.0), ("cfl", 0.0)):
        p = gks.params()
        setattr(p, field, value)
        assert gks.lib().gks_workspace_bytes(g._h, C.byref(p)) == 0, field
    # unknown boundary kinds are refused, the known ones (open .. moving wall) accepted
    gb = gks.Mesh(I.box_mesh((3, 2, 2), (1.0, 0.5, 0.5), (False, True, True), jitter=0.1, seed=5))
    kinds = np.zeros((gb.nc, 4), np.int8)
    for k in range(6):
        kinds[:] = k
        gb.set_boundary(kinds)
    kinds[:] = 6
    with pytest.raises(gks.GksError) as e:
        gb.set_boundary(kinds)
    assert e.value.status == -1


def test_batch_connectivity_matches_each_case(built, oracle_mod):
    """A batch is the disjoint union of its cases: per case, the connectivity
    equals the oracle's for that case alone (cell ids offset by the case's
    first cell); faces never join cells of different cases."""
    batch, W, dW, desc, meshes = I.batch_cases(n_cases=4, n_range=(2, 4), seed=3)
    g = gks.Mesh(batch)
    assert g.ncase == 4 and g.case_first[-1] == g.nc
    top = g.topology()
    for k, m in enumerate(meshes):
        to = oracle_mod.Mesh(m).topology()
        c0, c1 = g.case_first[k], g.case_first[k + 1]
        nb = top["nbr"][c0:c1]
        np.testing.assert_array_equal(np.where(nb >= 0, nb - c0, nb), to["nbr"])
        np.testing.assert_array_equal(top["csr_sign"][c0:c1], to["csr_sign"])
    lr = top["face_lr"]
    case_of = np.searchsorted(g.case_first, np.arange(g.nc), side="right") - 1
    assert (case_of[lr[:, 0]] == case_of[lr[:, 1]]).all()
    # cases must be grouped in ascending order
    bad = dict(batch)
    bad["case"] = batch["case"][::-1].copy()
    with pytest.raises(gks.GksError):
        gks.Mesh(bad)


def test_empty_mesh_is_rejected(built):
    mesh = {"xyz": np.zeros((0, 3)), "tet": np.zeros((0, 4), np.int64), "shift": np.zeros((0, 4, 3), np.int8),
            "period": np.zeros(3)}
    with pytest.raises(gks.GksError) as e:
        gks.Mesh(mesh)
    assert e.value.status == -1


def test_mesh_errors_found_on_worker_threads_reach_the_caller(built):
    """Mesh set-up splits its loops over the host's threads (48,000 cells
    here, so the last cells belong to a worker); a fault found there must
    come back as GKS_E_MESH with its message on the calling thread."""
    mesh = I.box_mesh((20, 20, 20), jitter=0.1, seed=6)
    nc = mesh["tet"].shape[0]
    # a tetrahedron that repeats a vertex id, in the last cell
    bad = dict(mesh)
    tet = mesh["tet"].copy()
    tet[nc - 1, 3] = tet[nc - 1, 0]
    bad["tet"] = tet
    with pytest.raises(gks.GksError) as e:
        gks.Mesh(bad)
    assert e.value.status == -2 and "repeats a vertex" in str(e.value)
    # a duplicated last cell: each of its faces is shared by three cells
    bad = dict(mesh)
    bad["tet"] = np.concatenate([mesh["tet"], mesh["tet"][-1:]])
    bad["shift"] = np.concatenate([mesh["shift"], mesh["shift"][-1:]])
    with pytest.raises(gks.GksError) as e:
        gks.Mesh(bad)
    assert e.value.status == -2 and "more than two cells" in str(e.value)
    # and the intact mesh still builds, every local face in the face list
    g = gks.Mesh(mesh)
    top = g.topology()
    assert g.nf == 2 * nc and (top["csr_face"] >= 0).all()
    assert np.bincount(top["csr_face"].ravel(), minlength=g.nf).tolist() == [2] * g.nf
