"""Partition-ready layout (Sec. 3.5) on the host, no GPU: recursive coordinate
bisection of the elements and, per part, the element list, owned faces,
interface faces and matvec halo, bit-exact against lists built here from the
oracle's connectivity; then two gloo ranks carry out the exchanges the layout
describes (interface rows of the condensed blocks to their owner, halo trace
entries for the matvec) on the oracle's element matrices and reproduce the
single-process assembly and matvec row by row."""
import os
import socket

import numpy as np
import pytest

import synth
from oracle import tet as ot
from oracle.mesh import Connectivity
from synth import tetmesh as tm

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


@pytest.fixture(scope="module")
def H():
    from paper_2608_27863_gb300 import build, hdg
    build.build()
    hdg.lib()
    return hdg


def hex_case(H, periodic=(True, False, True), n=(5, 3, 4)):
    mesh = synth.box_mesh(3, n, (0.0, 0.0, 0.0), (2.5, 1.0, 1.6), periodic)
    h = H.hdg_create(3, mesh.vert_xyz, mesh.elem_vert, mesh.periodic_map, mesh.bnd_tag, 1, 1.4, 100.0, 0.72, 0.3,
                     host_only=True)
    conn = Connectivity(mesh, 1)
    f2e = np.array(conn.f2e[:, :, 0])
    cen = mesh.vert_xyz[mesh.elem_vert].mean(axis=1)
    return h, f2e, np.asarray(conn.rowptr), np.asarray(conn.col), cen


def quad_case(H):
    mesh = synth.box_mesh(2, (7, 4), (0.0, 0.0), (1.4, 0.5), (True, False))
    h = H.hdg_create(2, mesh.vert_xyz, mesh.elem_vert, mesh.periodic_map, mesh.bnd_tag, 2, 1.4, 100.0, 0.72, 0.3,
                     host_only=True)
    conn = Connectivity(mesh, 2)
    f2e = np.array(conn.f2e[:, :, 0])
    cen = mesh.vert_xyz[mesh.elem_vert].mean(axis=1)
    return h, f2e, np.asarray(conn.rowptr), np.asarray(conn.col), cen


def tet_mesh():
    c = [np.linspace(0, 1, 3), np.linspace(0, 0.5, 3), np.linspace(0, 0.5, 2)]
    return tm.kuhn_box((2, 2, 1), c, (False, False, False), bump=tm.wall_bump(0.05), curved_layers=1, seed=3)


def tet_case(H):
    mesh = tet_mesh()
    h = H.hdg_create_tet(mesh.vert_xyz, mesh.elem_vert, mesh.periodic_map, mesh.bnd_tag, mesh.elem_p, mesh.geo,
                         1.4, 1e5, 0.72, 0.5, host_only=True)
    conn = ot.TetConnectivity(mesh)
    f2e = np.array(conn.f2e[:, :, 0])
    cen = mesh.vert_xyz[mesh.elem_vert].mean(axis=1)
    return h, f2e, np.asarray(conn.rowptr), np.asarray(conn.col), cen


def expected_layout(part, q, f2e, rowptr, col):
    """The layout of part q written out from its definition."""
    side = [np.where(f2e[:, s] >= 0, part[np.maximum(f2e[:, s], 0)], -1) for s in (0, 1)]
    p0 = side[0]
    p1 = np.where(side[1] >= 0, side[1], p0)
    owner = np.minimum(p0, p1)
    iface = np.nonzero((p0 != p1) & ((p0 == q) | (p1 == q)))[0]
    peer = np.where(p0[iface] == q, p1[iface], p0[iface])
    touched = np.zeros(len(part), bool)
    cross = np.nonzero(p0 != p1)[0]
    touched[f2e[cross, 0]] = True
    touched[f2e[cross, 1]] = True
    mine = np.nonzero(part == q)[0]
    elems = np.concatenate([mine[~touched[mine]], mine[touched[mine]]])
    faces = np.nonzero(owner == q)[0]
    halo = sorted({int(col[b]) for F in faces for b in range(rowptr[F], rowptr[F + 1]) if owner[col[b]] != q})
    return {"elems": elems, "faces": faces, "interface_faces": iface, "interface_peer": peer,
            "halo_faces": np.array(halo, np.int64), "halo_owner": owner[np.array(halo, np.int64)]}, owner


@pytest.mark.parametrize("n_parts", [1, 2, 3, 5, 8])
def test_partition_balanced_and_cut_along_longest_extent(H, n_parts):
    h, f2e, rowptr, col, cen = hex_case(H)
    try:
        part = H.hdg_partition(h, n_parts)
    finally:
        H.hdg_destroy(h)
    E = len(cen)
    counts = np.bincount(part, minlength=n_parts)
    assert np.array_equal(counts, [E // n_parts + (q < E % n_parts) for q in range(n_parts)])
    if n_parts > 1:        # the first cut: x has the longest extent; parts of the first half lie left of it
        left = np.isin(part, np.arange(n_parts // 2))
        assert cen[left, 0].max() <= cen[~left, 0].min()


@pytest.mark.parametrize("case", ["hex-periodic", "hex-box", "quad", "tet"])
@pytest.mark.parametrize("n_parts", [2, 3, 4])
def test_part_layout_bit_exact(H, case, n_parts):
    if case == "tet":
        h, f2e, rowptr, col, cen = tet_case(H)
    elif case == "quad":
        h, f2e, rowptr, col, cen = quad_case(H)
    else:
        h, f2e, rowptr, col, cen = hex_case(H, periodic=(True, False, True) if case == "hex-periodic"
                                            else (False, False, False))
    try:
        part = H.hdg_partition(h, n_parts)
        lays = [H.hdg_part_layout(h, part, q) for q in range(n_parts)]
    finally:
        H.hdg_destroy(h)
    for q, lay in enumerate(lays):
        exp, owner = expected_layout(part, q, f2e, rowptr, col)
        for k, v in exp.items():
            assert np.array_equal(lay[k], v), (q, k)
        s = lay["sizes"]
        assert s["n_interior_elem"] == int(np.sum(~np.isin(lay["elems"], f2e[lay["interface_faces"]].ravel())))
        assert s["n_elem"] == len(lay["elems"]) and s["n_halo_faces"] == len(lay["halo_faces"])
    # the parts cover elements and faces exactly once; interfaces are reciprocal
    assert np.array_equal(np.sort(np.concatenate([l["elems"] for l in lays])), np.arange(len(part)))
    assert np.array_equal(np.sort(np.concatenate([l["faces"] for l in lays])), np.arange(len(f2e)))
    pairs = sorted((int(F), min(q, int(r)), max(q, int(r))) for q, l in enumerate(lays)
                   for F, r in zip(l["interface_faces"], l["interface_peer"]))
    assert all(pairs[2 * i] == pairs[2 * i + 1] for i in range(len(pairs) // 2)) and len(pairs) % 2 == 0


def test_partition_argument_errors(H):
    h, f2e, rowptr, col, cen = hex_case(H)
    try:
        for bad in (0, len(cen) + 1):
            with pytest.raises(H.HDGError) as ex:
                H.hdg_partition(h, bad)
            assert ex.value.code == H.HDG_EINVAL
        with pytest.raises(H.HDGError):
            H.hdg_part_layout(h, -np.ones(len(cen), np.int32), 0)
    finally:
        H.hdg_destroy(h)


# ----------------------------------------------------------------------------
# two gloo ranks: assembly and matvec through the exchanges the layout names
# ----------------------------------------------------------------------------
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _tet_problem():
    mesh = tet_mesh()
    prob = tm.config4_problem(mesh)
    conn = ot.TetConnectivity(mesh)
    fun = tm.sinusoids(prob.gamma, prob.mach, 3, 1e-3)
    prob.U, prob.Q, prob.UH, prob.Ustar = tm.packed_state(mesh, fun, conn.nfp, prob.ubc, 5)
    return mesh, ot.TetProblem(prob)


def _row_width(c, F):
    return sum(int(c.hoff[c.col[b] + 1] - c.hoff[c.col[b]]) for b in range(c.rowptr[F], c.rowptr[F + 1]))


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2608_27863_gb300 import hdg as H
    mesh, pb = _tet_problem()
    c = pb.conn
    h = H.hdg_create_tet(mesh.vert_xyz, mesh.elem_vert, mesh.periodic_map, mesh.bnd_tag, mesh.elem_p, mesh.geo,
                         1.4, 1e5, 0.72, 0.5, host_only=True)
    part = H.hdg_partition(h, world)
    lays = [H.hdg_part_layout(h, part, r) for r in range(world)]
    H.hdg_destroy(h)
    me, peer = lays[rank], lays[1 - rank]
    # element-local work: condensed blocks of this part's elements, by block row
    rows = {}
    for e in me["elems"]:
        S = pb.condense(int(e))["S"]
        o = pb.element_trace_offsets(int(e))
        for fl, F in enumerate(c.e2f[e]):
            R = rows.setdefault(int(F), {})
            for gl, G in enumerate(c.e2f[e]):
                blk = S[o[fl]:o[fl + 1], o[gl]:o[gl + 1]]
                R[int(G)] = R.get(int(G), 0.0) + blk

    def pack(F, R):                     # row F as [bs_F][row width], blocks in column order, zeros if absent
        bsF = int(c.hoff[F + 1] - c.hoff[F])
        return np.concatenate([np.asarray(R.get(int(G), np.zeros((bsF, int(c.hoff[G + 1] - c.hoff[G])))))
                               for G in c.col[c.rowptr[F]:c.rowptr[F + 1]]], axis=1)

    # assembly exchange: interface rows go to their owner
    send = [F for F, r in zip(me["interface_faces"], me["interface_peer"]) if min(rank, r) != rank]
    recv = [F for F, r in zip(me["interface_faces"], me["interface_peer"]) if min(rank, r) == rank]
    req = None
    if send:
        req = dist.isend(torch.from_numpy(np.concatenate([pack(int(F), rows[int(F)]).ravel() for F in send])),
                         1 - rank)
    if recv:
        n = sum(int(c.hoff[F + 1] - c.hoff[F]) * _row_width(c, int(F)) for F in recv)
        buf = torch.zeros(n, dtype=torch.float64)
        dist.recv(buf, 1 - rank)
        off = 0
        for F in recv:
            F = int(F)
            own = pack(F, rows.get(F, {}))
            add = buf[off:off + own.size].numpy().reshape(own.shape)
            off += own.size
            rows[F] = {"packed": own + add}
    if req is not None:
        req.wait()
    owned = {int(F): (rows[int(F)]["packed"] if "packed" in rows[int(F)] else pack(int(F), rows[int(F)]))
             for F in me["faces"]}
    # matvec: x lives with the owners; each part receives its halo
    x = np.sin(0.37 * np.arange(c.hoff[-1])) + 0.2
    xl = {int(F): x[c.hoff[F]:c.hoff[F + 1]] for F in me["faces"]}
    out = [F for F, o in zip(peer["halo_faces"], peer["halo_owner"]) if o == rank]
    req = None
    if out:
        req = dist.isend(torch.from_numpy(np.concatenate([xl[int(F)] for F in out])), 1 - rank)
    if len(me["halo_faces"]):
        n = int(sum(c.hoff[F + 1] - c.hoff[F] for F in me["halo_faces"]))
        buf = torch.zeros(n, dtype=torch.float64)
        dist.recv(buf, 1 - rank)
        off = 0
        for F in me["halo_faces"]:
            k = int(c.hoff[F + 1] - c.hoff[F])
            xl[int(F)] = buf[off:off + k].numpy()
            off += k
    if req is not None:
        req.wait()
    y = {F: owned[F] @ np.concatenate([xl[int(G)] for G in c.col[c.rowptr[F]:c.rowptr[F + 1]]]) for F in owned}
    dist.barrier()
    q.put((rank, {F: owned[F] for F in owned}, y, len(send), len(out)))
    dist.destroy_process_group()


def test_two_gloo_ranks_assemble_and_apply_through_the_layout(H):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    mesh, pb = _tet_problem()
    c = pb.conn
    vals, _ = pb.assemble()
    x = np.sin(0.37 * np.arange(c.hoff[-1])) + 0.2
    yref = pb.matvec(vals, x)
    seen = set()
    assert res[1][3] > 0 and res[0][4] + res[1][4] > 0      # rank 1 sent interface rows; halos were exchanged
    for rank, owned, y, _, _ in res:
        for F, row in owned.items():
            ref = np.concatenate([vals[b] for b in range(c.rowptr[F], c.rowptr[F + 1])], axis=1)
            assert np.allclose(row, ref, rtol=0, atol=1e-12 * np.abs(ref).max()), (rank, F)
            yr = yref[c.hoff[F]:c.hoff[F + 1]]
            assert np.allclose(y[F], yr, rtol=0, atol=1e-12 * np.abs(yref).max()), (rank, F)
            seen.add(F)
    assert seen == set(range(c.n_faces))
