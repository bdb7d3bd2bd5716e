"""The C-ABI library without a GPU: symbols, host set-up, integer connectivity.

Integer outputs (face-to-element maps, orientation permutations, block-sparse
pattern) are compared bit-exactly with the oracle's independent implementation.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from oracle.mesh import Connectivity

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    from paper_2608_27863_gb300 import build, hdg
    build.build()
    hdg.lib()
    return hdg


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hdg.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(hdg_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol(H):
    syms = declared_symbols()
    assert len(syms) >= 14
    L = ctypes.CDLL(H.LIB_PATH)
    for s in syms:
        assert hasattr(L, s), s
    assert sorted(H.EXPORTS) == syms


def test_connectivity_bit_exact_with_boundaries(H):
    for dim, per in ((2, (True, False)), (3, (True, False, True)), (3, (False, False, False))):
        mesh = synth.box_mesh(dim, (3, 4, 3)[:dim], (0,) * dim, (1.0,) * dim, per)
        h = H.hdg_create_host(dim, mesh.vert_xyz, mesh.elem_vert, mesh.periodic_map, mesh.bnd_tag, 2,
                              1.4, 100.0, 0.72, 0.3)
        c = H.hdg_get_connectivity(h)
        H.hdg_destroy(h)
        o = Connectivity(mesh, 2)
        assert np.array_equal(c["f2e"], o.f2e[:, :, 0]) and np.array_equal(c["f2lf"], o.f2e[:, :, 1])
        assert np.array_equal(c["perm"], o.perm) and np.array_equal(c["col"], o.col)
        assert np.array_equal(c["rowptr"], o.rowptr)


def test_boundary_tag_checks(H):
    mesh = synth.box_mesh(2, (3, 3), (0, 0), (1, 1), (True, False))
    bad = mesh.bnd_tag.copy()
    bad[bad == 1] = 7
    with pytest.raises(H.HDGError) as ex:
        H.hdg_create_host(2, mesh.vert_xyz, mesh.elem_vert, mesh.periodic_map, bad, 2, 1.4, 100.0, 0.72, 0.3)
    assert ex.value.code == H.HDG_EUNSUPPORTED
    for t in (2, 3, 4):                     # outflow, isothermal and adiabatic walls are accepted
        ok = mesh.bnd_tag.copy()
        ok[ok == 1] = t
        H.hdg_destroy(H.hdg_create_host(2, mesh.vert_xyz, mesh.elem_vert, mesh.periodic_map, ok, 2, 1.4, 100.0,
                                        0.72, 0.3))
    inner = mesh.bnd_tag.copy()
    inner[4, 0] = 3                         # an interior face marked as a wall
    with pytest.raises(H.HDGError) as ex:
        H.hdg_create_host(2, mesh.vert_xyz, mesh.elem_vert, mesh.periodic_map, inner, 2, 1.4, 100.0, 0.72, 0.3)
    assert ex.value.code == H.HDG_EINVAL
    with pytest.raises(H.HDGError) as ex:   # boundary faces without tags
        H.hdg_create_host(2, mesh.vert_xyz, mesh.elem_vert, mesh.periodic_map, None, 2, 1.4, 100.0, 0.72, 0.3)
    assert ex.value.code == H.HDG_EINVAL


def mesh_cases():
    cases = []
    for dim, n in ((2, (3, 4)), (3, (3, 3, 4))):
        for p in (1, 2, 3):
            cases.append((dim, n, p, False))
    cases.append((3, (3, 3, 3), 2, True))
    cases.append((2, (4, 3), 3, True))
    return cases


@pytest.mark.parametrize("dim,n,p,scramble", mesh_cases())
def test_connectivity_bit_exact(H, dim, n, p, scramble):
    mesh = synth.box_mesh(dim, n, (0,) * dim, (1.0,) * dim, (True,) * dim)
    if scramble:
        rng = np.random.default_rng(11)
        perm = rng.permutation(mesh.n_vert)
        inv = np.argsort(perm)
        mesh.vert_xyz = mesh.vert_xyz[inv]
        mesh.elem_vert = perm[mesh.elem_vert]
        mesh.periodic_map = perm[mesh.periodic_map[inv]]
    h = H.hdg_create_host(dim, mesh.vert_xyz, mesh.elem_vert, mesh.periodic_map, None, p, 1.4, 100.0, 0.72, 0.3)
    c = H.hdg_get_connectivity(h)
    H.hdg_destroy(h)
    o = Connectivity(mesh, p)
    assert c["f2e"].shape[0] == o.n_faces
    assert np.array_equal(c["f2e"], o.f2e[:, :, 0])
    assert np.array_equal(c["f2lf"], o.f2e[:, :, 1])
    assert np.array_equal(c["e2f"], o.e2f)
    assert np.array_equal(c["perm"], o.perm)
    assert np.array_equal(c["rowptr"], o.rowptr)
    assert np.array_equal(c["col"], o.col)


def test_argument_errors(H):
    mesh = synth.box_mesh(2, (3, 3), (0, 0), (1, 1), (True, True))
    args = (2, mesh.vert_xyz, mesh.elem_vert, mesh.periodic_map, None)
    with pytest.raises(H.HDGError) as ex:
        H.hdg_create_host(*args, 4, 1.4, 100.0, 0.72, 0.3)
    assert ex.value.code == H.HDG_EUNSUPPORTED
    with pytest.raises(H.HDGError) as ex:
        H.hdg_create_host(*args, 2, 0.9, 100.0, 0.72, 0.3)
    assert ex.value.code == H.HDG_EINVAL
    # a non-affine (trapezoidal) element
    xyz = mesh.vert_xyz.copy()
    xyz[5, 0] += 0.05
    with pytest.raises(H.HDGError) as ex:
        H.hdg_create_host(2, xyz, mesh.elem_vert, mesh.periodic_map, None, 2, 1.4, 100.0, 0.72, 0.3)
    assert ex.value.code == H.HDG_EUNSUPPORTED
    # an element on both sides of a periodic face (one element across)
    short = synth.box_mesh(2, (3, 3), (0, 0), (1, 1), (True, True))
    pm = short.periodic_map.copy()
    pm[1] = 0  # identify x = 1/3 with x = 0: element 0 sees itself
    with pytest.raises(H.HDGError) as ex:
        H.hdg_create_host(2, short.vert_xyz, short.elem_vert, pm, None, 2, 1.4, 100.0, 0.72, 0.3)
    assert ex.value.code == H.HDG_EINVAL
    # device calls on a host-only handle
    h = H.hdg_create_host(*args, 2, 1.4, 100.0, 0.72, 0.3)
    rc = H.lib().hdg_trace_matvec(h, None, None)
    assert rc == H.HDG_EINVAL
    assert "assembled" in H.hdg_last_error(h) or "device" in H.hdg_last_error(h)
    H.hdg_destroy(h)


def test_empty_and_degenerate_meshes(H):
    mesh = synth.box_mesh(2, (3, 3), (0, 0), (1, 1), (True, True))
    empty = np.zeros((0, 4), dtype=np.int64)
    with pytest.raises(H.HDGError) as ex:          # no elements
        H.hdg_create_host(2, mesh.vert_xyz, empty, mesh.periodic_map, None, 2, 1.4, 100.0, 0.72, 0.3)
    assert ex.value.code == H.HDG_EINVAL
    flat = mesh.vert_xyz.copy()
    flat[:, 1] = 0.0                                # zero-area elements
    with pytest.raises(H.HDGError) as ex:
        H.hdg_create_host(2, flat, mesh.elem_vert, mesh.periodic_map, None, 2, 1.4, 100.0, 0.72, 0.3)
    assert ex.value.code in (H.HDG_EINVAL, H.HDG_EUNSUPPORTED)
    bad = mesh.elem_vert.copy()
    bad[0, 0] = mesh.n_vert + 5                     # vertex index out of range
    with pytest.raises(H.HDGError) as ex:
        H.hdg_create_host(2, mesh.vert_xyz, bad, mesh.periodic_map, None, 2, 1.4, 100.0, 0.72, 0.3)
    assert ex.value.code == H.HDG_EINVAL


def test_single_element_thick_mesh_is_rejected_or_consistent(H):
    """An open box of one element (all faces boundary) is a valid mesh: four boundary faces."""
    mesh = synth.box_mesh(2, (1, 1), (0, 0), (1, 1), (False, False))
    h = H.hdg_create_host(2, mesh.vert_xyz, mesh.elem_vert, mesh.periodic_map, mesh.bnd_tag, 1, 1.4, 100.0, 0.72,
                          0.3)
    c = H.hdg_get_connectivity(h)
    H.hdg_destroy(h)
    assert c["f2e"].shape[0] == 4 and np.all(c["f2e"][:, 1] == -1)
    assert np.array_equal(c["rowptr"], [0, 4, 8, 12, 16])


def test_sdirk3_tableau_from_the_library(H):
    """The library's SDIRK3 (gamma from the L-stability cubic) against the oracle's
    (gamma from the third-order condition): the same tableau; the binding only
    marshals it."""
    from oracle.dirk import alexander_sdirk3
    A, b = H.sdirk3_tableau()
    Ao, bo, _ = alexander_sdirk3()
    assert np.allclose(A, Ao, rtol=0, atol=1e-14) and np.allclose(b, bo, rtol=0, atol=1e-14)
    assert np.array_equal(b, A[-1])
    c = A.sum(1)
    assert abs(b @ c ** 2 - 1 / 3) < 1e-14 and abs(b @ A @ c - 1 / 6) < 1e-14
