"""Host side of the tetrahedral path without a GPU: reference tables, skeleton,
face degrees, canonical frames and the variable-size block layout, against the
oracle (tables to rounding, integers bit-exact)."""
import numpy as np
import pytest

from oracle import tet as ot
from synth import tetmesh as tm


@pytest.fixture(scope="module")
def H():
    from paper_2608_27863_gb300 import build, hdg
    build.build()
    hdg.lib()
    return hdg


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_reference_tables_match_oracle(H, p):
    t, r = H.hdg_tet_ref_tables(p), ot.TetRef(p)
    assert np.allclose(t["xq"], r.xq, atol=1e-15, rtol=0)
    assert np.allclose(t["wq"], r.wq, atol=1e-15, rtol=0)
    assert np.allclose(t["phi"], r.phi, atol=1e-13, rtol=0)
    assert np.allclose(t["dphi"], r.dphi, atol=1e-12, rtol=0)
    tt, T = H.hdg_tri_ref_tables(p), ot.TriRef(p)
    assert np.allclose(tt["xs"], T.xs, atol=1e-15, rtol=0)
    assert np.allclose(tt["ws"], T.ws, atol=1e-15, rtol=0)
    assert np.allclose(tt["mu"], T.mu, atol=1e-13, rtol=0)


def meshes():
    c3 = [np.linspace(0, 1, 4), np.linspace(0, 0.5, 3), np.linspace(0, 0.75, 4)]
    return [
        tm.kuhn_box((2, 1, 1), [np.linspace(0, 1, 3), np.linspace(0, .5, 2), np.linspace(0, .5, 2)],
                    (False, False, False), bump=tm.wall_bump(0.05), curved_layers=1, seed=3),
        tm.kuhn_box((3, 2, 3), c3, (True, False, True), tags={(1, 0): 4, (1, 1): 1}, bump=tm.wall_bump(0.05),
                    curved_layers=1, seed=5),
        tm.kuhn_box((3, 3, 3), [np.linspace(0, 1, 4)] * 3, (True, True, True), degrees=2, seed=1),
    ]


@pytest.mark.parametrize("k", [0, 1, 2])
def test_layout_bit_exact(H, k):
    mesh = meshes()[k]
    h = H.hdg_create_tet(mesh.vert_xyz, mesh.elem_vert, mesh.periodic_map, mesh.bnd_tag, mesh.elem_p, mesh.geo,
                         1.4, 1e5, 0.72, 0.5, host_only=True)
    try:
        L = H.hdg_tet_layout(h)
        s = H.hdg_tet_query(h)
    finally:
        H.hdg_destroy(h)
    o = ot.TetConnectivity(mesh)
    assert s["n_faces"] == o.n_faces and s["nnzb"] == len(o.col)
    assert np.array_equal(L["f2e"], o.f2e[:, :, 0])
    assert np.array_equal(L["e2f"], o.e2f)
    assert np.array_equal(L["frame"], o.L)
    assert np.array_equal(L["face_p"], o.face_p)
    assert np.array_equal(L["hoff"], o.hoff) and np.array_equal(L["uoff"], o.uoff)
    assert np.array_equal(L["rowptr"], o.rowptr) and np.array_equal(L["col"], o.col)
    assert np.array_equal(L["boff"], o.boff)
    assert s["n_trace"] == o.hoff[-1] and s["n_u"] == o.uoff[-1] and s["n_vals"] == o.boff[-1]
    curved = sum(1 for e in range(mesh.n_elem)
                 if np.abs(mesh.geo[e, 4:] - 0.5 * (mesh.geo[e, [0, 0, 0, 1, 1, 2]] +
                                                    mesh.geo[e, [1, 2, 3, 2, 3, 3]])).max() > 1e-12)
    assert s["n_curved"] == curved


def test_tet_argument_errors(H):
    mesh = meshes()[0]
    args = (mesh.vert_xyz, mesh.elem_vert, mesh.periodic_map, mesh.bnd_tag)
    bad = mesh.elem_p.copy()
    bad[0] = 5
    with pytest.raises(H.HDGError) as ex:
        H.hdg_create_tet(*args, bad, mesh.geo, 1.4, 1e5, 0.72, 0.5, host_only=True)
    assert ex.value.code == H.HDG_EUNSUPPORTED
    with pytest.raises(H.HDGError) as ex:                 # untagged boundary faces
        H.hdg_create_tet(mesh.vert_xyz, mesh.elem_vert, mesh.periodic_map, None, mesh.elem_p, mesh.geo,
                         1.4, 1e5, 0.72, 0.5, host_only=True)
    assert ex.value.code == H.HDG_EINVAL
    inv = mesh.elem_vert.copy()
    inv[:, [1, 2]] = inv[:, [2, 1]]                       # negative orientation
    with pytest.raises(H.HDGError) as ex:
        H.hdg_create_tet(mesh.vert_xyz, inv, mesh.periodic_map, mesh.bnd_tag, mesh.elem_p, None,
                         1.4, 1e5, 0.72, 0.5, host_only=True)
    assert ex.value.code == H.HDG_EINVAL
    h = H.hdg_create_tet(*args, mesh.elem_p, mesh.geo, 1.4, 1e5, 0.72, 0.5, host_only=True)
    try:                                                   # hex-only entry points refuse tetrahedral handles
        assert H.lib().hdg_lift_gradient(h, None, None, None) == H.HDG_EUNSUPPORTED
        assert H.lib().hdg_reserve(h, 0) == H.HDG_EUNSUPPORTED
        assert H.lib().hdg_set_preconditioner(h, H.HDG_PC_SCHWARZ) == H.HDG_OK   # patches of mixed size
        assert H.lib().hdg_schwarz_setup(h) == H.HDG_EINVAL                       # nothing assembled on the host
    finally:
        H.hdg_destroy(h)
