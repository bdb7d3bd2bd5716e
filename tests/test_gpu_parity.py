"""GPU FP64 path vs the FP64 oracle, element by element and block by block.

Bar: every compared block of the assembled trace matrix within 1e-11 relative
Frobenius norm, the condensed right-hand side and the recovered interior
corrections within 1e-11 relative to their norm; integer data bit-exact
(tested on the host in test_lib_host.py).  Small meshes are compared in full;
the full-size workloads on sampled block rows (the two elements of each
sampled face provide every contribution to the row).
"""
import os

import numpy as np
import pytest

import synth
from oracle.hdg import Problem
from tests.helpers import GpuRun, block_rel_errors, create

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_27863_gb300 import build
    build.build()


def compare(P, rows=None, check_matvec=False, seed=0, tuning=None):
    from paper_2608_27863_gb300 import hdg as H
    run = GpuRun(P)
    if tuning:
        H.hdg_set_tuning(run.h, **tuning)
    run.linearize()
    assert H.hdg_status(run.h) == 0
    vals = run.blocks()
    g = run.rhs()
    pb = Problem(P)
    cn = pb.conn
    rows = range(cn.n_faces) if rows is None else rows
    blocks = [b for F in rows for b in range(cn.rowptr[F], cn.rowptr[F + 1])]
    orc, cache = pb.assemble(blocks=blocks)
    errs = block_rel_errors(vals, orc)
    worst = max(errs.values())
    assert worst < TOL, worst
    og = pb.assemble_g(cache, rows)
    for F in rows:
        assert np.linalg.norm(g[F] - og[F]) <= TOL * max(np.linalg.norm(og[F]), 1e-300), F
    rng = np.random.default_rng(seed)
    dUH = rng.normal(size=P.UH.shape) * np.abs(P.UH).mean(axis=(0, 2))[None, :, None] * 1e-3
    dQ, dU = run.recover(dUH)
    for e in sorted(cache):
        oq, ou = pb.recover(e, cache[e], dUH)
        assert np.linalg.norm(dU[e] - ou) <= TOL * np.linalg.norm(ou), e
        assert np.linalg.norm(dQ[e] - oq) <= TOL * np.linalg.norm(oq), e
    if check_matvec:
        x = rng.normal(size=P.UH.shape)
        y = run.matvec(x)
        # kernel alone: against a dense product with the GPU's own blocks
        bs = vals.shape[1]
        xv = x.reshape(cn.n_faces, bs)
        yref = np.zeros_like(xv)
        for F in range(cn.n_faces):
            for b in range(cn.rowptr[F], cn.rowptr[F + 1]):
                yref[F] += vals[b] @ xv[cn.col[b]]
        assert np.abs(y.reshape(yref.shape) - yref).max() <= 1e-13 * np.abs(yref).max()
        # whole path: against the oracle's assembled operator
        yo = pb.matvec(orc, x)
        assert np.linalg.norm(y - yo) <= TOL * np.linalg.norm(yo)
    run.close()
    return worst


def test_config1_quad_p2_full():
    """8 x 8 periodic unit square, quads p = 2 (the small workload), everything compared."""
    compare(synth.config1(), check_matvec=True)


@pytest.mark.parametrize("dim,p,law,av", [(2, 1, 0, 0.0), (2, 3, 1, 2e-3), (3, 1, 1, 1e-3)])
def test_tiny_meshes_full(dim, p, law, av):
    compare(synth.tiny(dim, p, visc_law=law, av=av), check_matvec=True)


def test_hex_p2_small_full():
    """3 x 3 x 3 TGV hexes p = 2: several tiles of every kernel, ragged tails."""
    compare(synth.config2(n=3), check_matvec=True)


def test_hex_p3_small_sampled():
    P = synth.config3(n=3)
    compare(P, rows=[0, 17, 40])


def test_skewed_scrambled_nonuniform_mesh():
    """Parallelepiped elements, a 3 x 4 x 3 box and randomly relabelled vertices
    (rotated / reflected face frames)."""
    P = synth.config_tgv(3, 2, 0.5, 5, True, 1e-3)
    mesh = synth.box_mesh(3, (3, 4, 3), (0,) * 3, (2 * np.pi,) * 3, (True,) * 3)
    rng = np.random.default_rng(4)
    perm = rng.permutation(mesh.n_vert)
    inv = np.argsort(perm)
    xyz = mesh.vert_xyz[inv].copy()
    xyz[:, 0] += 0.2 * xyz[:, 1] + 0.1 * xyz[:, 2]
    xyz[:, 2] += 0.15 * xyz[:, 1]
    mesh.vert_xyz = xyz
    mesh.elem_vert = perm[mesh.elem_vert]
    mesh.periodic_map = perm[mesh.periodic_map[inv]]
    x = synth.node_xyz(mesh, 2)
    fun = lambda y: synth.tgv_state(y, 1.4, 0.5)
    P.mesh = mesh
    P.U = np.ascontiguousarray(fun(x).transpose(0, 2, 1))
    P.Q = np.ascontiguousarray(synth.nodal_gradient(fun, x).transpose(0, 2, 3, 1))
    P.Ustar = P.U + 1e-3 * synth.normal(9, P.U.size).reshape(P.U.shape)
    P.UH = P.UH[:mesh.n_faces()] if P.UH.shape[0] >= mesh.n_faces() else np.resize(P.UH, (mesh.n_faces(),) + P.UH.shape[1:])
    P.nu = synth.synthetic_nu(mesh, 2, 3, 1e-3)
    compare(P, rows=[0, 5, 33, 70, 107])


@pytest.mark.parametrize("dim,p,per", [(2, 2, (True, False)), (3, 1, (True, False, True)), (2, 3, (False, False))])
def test_dirichlet_boundary_faces(dim, p, per):
    """Tag-1 faces (bhat = uhat - u_b): trace rows, assembly with one-sided faces."""
    compare(synth.tiny(dim, p, periodic=per, visc_law=1, av=1e-3), check_matvec=True)


def test_chunking_is_bitwise_invisible():
    P = synth.config2(n=3)
    a = GpuRun(P).linearize()
    va, ga = a.blocks(), a.rhs()
    a.close()
    os.environ["HDG_SCRATCH_BYTES"] = str(5 * 1024 * 1024)   # a few elements per chunk, ragged last chunk
    try:
        b = GpuRun(P).linearize()
    finally:
        del os.environ["HDG_SCRATCH_BYTES"]
    vb, gb = b.blocks(), b.rhs()
    b.linearize()
    vc = b.blocks()
    b.close()
    assert np.array_equal(va, vb) and np.array_equal(ga, gb)
    assert np.array_equal(vb, vc)   # run-to-run determinism


def sampled_rows(P, seed, n):
    """n seeded face rows plus the faces of the first and last elements (which
    include faces identified across the periodic boundary)."""
    from oracle.mesh import Connectivity
    c = Connectivity(P.mesh, P.p)
    rows = {int(r) for r in synth.splitmix64(seed, n) % np.uint64(c.n_faces)}
    rows |= {int(F) for e in (0, P.mesh.n_elem - 1) for F in c.e2f[e]}
    return sorted(rows)


def test_config2_full_size_sampled():
    """16^3 = 4096 hexes p = 2, sampled block rows (24 seeded + 12 periodic-edge faces)."""
    P = synth.config2()
    compare(P, rows=sampled_rows(P, 21, 24))


def test_config3_full_size_sampled():
    """24^3 = 13824 hexes p = 3, Sutherland + artificial viscosity, sampled rows
    (10 seeded + 12 periodic-edge faces)."""
    P = synth.config3()
    compare(P, rows=sampled_rows(P, 22, 10))


def test_nonfinite_input_is_reported():
    import torch
    from paper_2608_27863_gb300 import hdg as H
    P = synth.tiny(2, 2)
    P.U = P.U.copy()
    P.U[4, 0, 3] = np.nan
    run = GpuRun(P).linearize()
    assert H.hdg_status(run.h) == H.HDG_ENONFINITE
    # the handle stays usable
    run.U.copy_(torch.from_numpy(synth.tiny(2, 2).U).cuda())
    run.linearize()
    assert H.hdg_status(run.h) == 0
    run.close()


@pytest.mark.parametrize("make", [synth.config1, lambda: synth.tiny(2, 3, periodic=(True, False)),
                                  lambda: synth.config2(n=3), lambda: synth.tiny(3, 1, periodic=(False, True, True))],
                         ids=["quad-p2", "quad-p3-dirichlet", "hex-p2", "hex-p1-dirichlet"])
def test_lift_gradient_matches_oracle(make):
    import torch
    from paper_2608_27863_gb300 import hdg as H
    P = make()
    run = GpuRun(P)
    Q = torch.full_like(run.Q, np.nan)
    H.hdg_lift_gradient(run.h, run.U, run.UH, Q)
    torch.cuda.synchronize()
    oq = Problem(P).lift_gradient(P.U, P.UH)
    q = Q.cpu().numpy()
    assert np.linalg.norm(q - oq) <= TOL * np.linalg.norm(oq)
    run.close()


def test_autotuned_variants_keep_parity():
    """Every FP64 elimination variant the autotuner may pick meets the parity bar."""
    from paper_2608_27863_gb300 import hdg as H
    P = synth.config2(n=3)
    run = GpuRun(P)
    rep = H.hdg_autotune(run.h, run.U, run.Q, run.UH, run.Ustar, run.nu, P.dt, P.a_ii, reps=1)
    cands = rep["candidates"]
    assert len(cands) == 16 and all(ms > 0 for _, ms in cands)
    chosen = (rep["elim_nb"], rep["elim_minb"], rep["schur_mode"], rep["blocks64_mode"])
    assert min(ms for _, ms in cands) == [ms for c, ms in cands if (c[0], c[1], c[2], c[5]) == chosen][0]
    assert {c[5] for c, _ in cands} == {0, 1}      # dense and sum-factorised contraction
    assert {c[2] for c, _ in cands} == {0, 3}      # Schur product on the FP64 pipe / the tensor cores
    run.close()
    for cand, _ms in cands:
        nb, minb = cand[0], cand[1]
        h = create(P)
        H.hdg_set_tuning(h, elim_nb=nb, elim_minb=minb, schur_mode=cand[2], blocks64_mode=cand[5])
        compare_handle = GpuRun(P, h)
        compare_handle.linearize()
        vals = compare_handle.blocks()
        pb = Problem(P)
        rows = [0, 40, 77]
        blocks = [b for F in rows for b in range(pb.conn.rowptr[F], pb.conn.rowptr[F + 1])]
        orc, _ = pb.assemble(blocks=blocks)
        assert max(block_rel_errors(vals, orc).values()) < TOL, cand
        compare_handle.close()


def tagged(P, side_tags, twall=1.0):
    bt = P.mesh.bnd_tag.copy()
    for (r, s), t in side_tags.items():
        col = bt[:, 2 * r + s]
        col[col != 0] = t
    P.mesh.bnd_tag = bt
    P.twall = twall
    return P


BOUNDARY_CASES = {
    "quad-p2-inflow-outflow": lambda: tagged(synth.tiny(2, 2, periodic=(False, True), visc_law=1, av=1e-3),
                                             {(0, 0): 1, (0, 1): 2}),
    "quad-p3-isothermal": lambda: tagged(synth.tiny(2, 3, periodic=(True, False), visc_law=1),
                                         {(1, 0): 3, (1, 1): 1}, twall=0.8),
    "quad-p1-adiabatic-box": lambda: tagged(synth.tiny(2, 1, periodic=False, av=2e-3),
                                            {(r, s): 4 for r in range(2) for s in (0, 1)}),
    "hex-p2-wall-channel": lambda: tagged(synth.tiny(3, 2, periodic=(True, False, True), visc_law=1),
                                          {(1, 0): 3, (1, 1): 4}, twall=1.2),
    "hex-p1-all-kinds": lambda: tagged(synth.tiny(3, 1, periodic=False, av=1e-3),
                                       {(0, 0): 1, (0, 1): 2, (1, 0): 3, (1, 1): 4, (2, 0): 3, (2, 1): 1}, twall=0.9),
}


@pytest.mark.parametrize("name", list(BOUNDARY_CASES))
def test_boundary_kinds(name):
    """Outflow and no-slip wall faces (tags 2-4) next to far-field faces: full comparison."""
    compare(BOUNDARY_CASES[name](), check_matvec=True)


def test_nodal_inflow_profile():
    """Tag-1 faces with nodal boundary data (an inflow profile) instead of a constant state."""
    P = tagged(synth.tiny(2, 2, periodic=(False, True)), {(0, 0): 1, (0, 1): 2})
    cn = Problem(P).conn
    ubc = np.broadcast_to(np.asarray(P.ubc)[None, :, None], (cn.n_faces, 4, 3)).copy()
    ubc[:, 1, :] *= 1.0 + 0.1 * synth.uniform(3, ubc[:, 1, :].size).reshape(ubc[:, 1, :].shape)
    P.ubc = ubc
    compare(P, check_matvec=True)


@pytest.mark.parametrize("dim,p", [(2, 3), (3, 2)])
def test_single_element_box(dim, p):
    """The degenerate mesh of one element whose faces are all boundary faces."""
    mesh = synth.box_mesh(dim, (1,) * dim, (0.0,) * dim, (1.0,) * dim, (False,) * dim)
    ub = synth.freestream(dim, 1.4, 0.5)
    fun = lambda x: synth.conserved(1.0 + 0.1 * np.sin(3 * x[..., 0]), [0.3 + 0.1 * x[..., 1]] +
                                    [0.05 * x[..., 0]] * (dim - 1), 2.857 + 0.1 * x[..., 0], 1.4)
    U, Q, UH, Ustar = synth._stage_state(mesh, p, fun, ub, 3, 1e-3, 1e-2, 1e-3)
    P = synth.Problem("one-element", mesh, p, 1.4, 50.0, 0.72, 0.5, 3.0, 5e-2, 0.4, 1, 1.4042, 0.40417,
                      U, Q, UH, Ustar, None, ub)
    compare(P, check_matvec=True)
