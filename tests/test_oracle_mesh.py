"""Pins of the oracle's skeleton connectivity (faces, orientation, BSR pattern)."""
import numpy as np
import pytest

import synth
from oracle.mesh import Connectivity
from oracle.refelem import RefElem


def _check_orientation(mesh, p, lengths):
    """Both sides of every face put canonical node k at the same physical point
    (up to one periodic shift per face), and canonical node 0 sits at the corner
    with the smallest master vertex id."""
    cn = Connectivity(mesh, p)
    ref = RefElem(mesh.dim, p)
    x = synth.node_xyz(mesh, p)
    for F in range(cn.n_faces):
        sides = [tuple(s) for s in cn.f2e[F] if s[0] >= 0]
        pos = []
        for (e, f) in sides:
            inv = np.argsort(cn.perm[e, f])
            assert sorted(cn.perm[e, f]) == list(range(ref.Nfp))
            pos.append(x[e, ref.fnode[f][inv]])          # canonical order
        if len(pos) == 2:
            shift = pos[1] - pos[0]
            assert np.allclose(shift, shift[0], atol=1e-12)
            for k in range(mesh.dim):
                s = shift[0, k]
                assert abs(s) < 1e-12 or abs(abs(s) - lengths[k]) < 1e-12
        # origin rule
        ids = cn.corner_ids[F]
        e, f = sides[0]
        inv = np.argsort(cn.perm[e, f])
        node0 = x[e, ref.fnode[f][inv[0]]]
        vmin = min(ids)
        cands = np.where(mesh.periodic_map == vmin)[0]
        assert any(np.allclose(node0 - mesh.vert_xyz[c], 0.0, atol=1e-12) or
                   all(abs(abs(dd) - L) < 1e-12 or abs(dd) < 1e-12 for dd, L in zip(node0 - mesh.vert_xyz[c], lengths))
                   for c in cands)
    return cn


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2), (3, 3)])
def test_periodic_box_orientation(dim, p):
    n = (3, 4, 5)[:dim]
    mesh = synth.box_mesh(dim, n, (0,) * dim, (1.0,) * dim, (True,) * dim)
    cn = _check_orientation(mesh, p, (1.0,) * dim)
    assert cn.n_faces == dim * mesh.n_elem == mesh.n_faces()
    assert all(s[1][0] >= 0 for s in cn.f2e)


def test_scrambled_vertex_ids_orientation():
    """Relabel vertices randomly so that face frames are rotated / reflected."""
    mesh = synth.box_mesh(3, (3, 3, 3), (0,) * 3, (1.0,) * 3, (True, False, True))
    rng = np.random.default_rng(5)
    perm = rng.permutation(mesh.n_vert)
    inv = np.argsort(perm)
    mesh.vert_xyz = mesh.vert_xyz[inv]
    mesh.elem_vert = perm[mesh.elem_vert]
    mesh.periodic_map = perm[mesh.periodic_map[inv]]
    _check_orientation(mesh, 3, (1.0, 1.0, 1.0))


@pytest.mark.parametrize("dim", [2, 3])
def test_bsr_pattern(dim):
    mesh = synth.box_mesh(dim, (3,) * dim, (0,) * dim, (1,) * dim, (True,) * dim)
    cn = Connectivity(mesh, 1)
    per_row = 2 * (2 * dim - 1) + 1
    for F in range(cn.n_faces):
        cols = cn.col[cn.rowptr[F]:cn.rowptr[F + 1]]
        assert list(cols) == sorted(set(cols)) and F in cols
        assert len(cols) == per_row
    # symmetric pattern; contributions sorted and consistent
    pairs = {(F, int(G)) for F in range(cn.n_faces) for G in cn.col[cn.rowptr[F]:cn.rowptr[F + 1]]}
    assert all((G, F) in pairs for (F, G) in pairs)
    for b, lst in enumerate(cn.contrib):
        assert [c[0] for c in lst] == sorted(c[0] for c in lst)
        F = int(np.searchsorted(cn.rowptr, b, side="right") - 1)
        assert len(lst) == (2 if cn.col[b] == F else 1)
