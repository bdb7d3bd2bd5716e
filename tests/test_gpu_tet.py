"""GPU parity of the tetrahedral path (mixed degree, quadratic geometry) against
the FP64 oracle: condensed blocks, right-hand side, trace matvec and interior
recovery, through the C-ABI.  Tolerance 1e-11 relative per block norm."""
import numpy as np
import pytest

from oracle import tet as ot
from synth import tetmesh as tm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def H():
    from paper_2608_27863_gb300 import build, hdg
    build.build()
    hdg.lib()
    return hdg


def mesh_case(k):
    if k == 0:       # all-boundary box, far field everywhere, curved, degrees 1..4
        return tm.kuhn_box((2, 1, 1), [np.linspace(0, 1, 3), np.linspace(0, .5, 2), np.linspace(0, .5, 2)],
                           (False, False, False), bump=tm.wall_bump(0.05), curved_layers=1, seed=3)
    if k == 1:       # periodic x, z; adiabatic wall below, far field above; curved wall layer + affine top
        c = [np.linspace(0, 1, 4), np.array([0.0, 0.02, 0.1]), np.linspace(0, 0.6, 4)]
        return tm.kuhn_box((3, 2, 3), c, (True, False, True), tags={(1, 0): 4, (1, 1): 1},
                           bump=tm.wall_bump(0.05), curved_layers=1, seed=6)
    # isothermal wall and supersonic outflow sides, straight-sided
    c = [np.linspace(0, 1, 3), np.linspace(0, 0.5, 2), np.linspace(0, 0.5, 3)]
    return tm.kuhn_box((2, 1, 2), c, (False, False, False), tags={(1, 0): 3, (0, 1): 2}, seed=9)


def setup(H, mesh, seed=5, twall=None):
    prob = tm.config4_problem(mesh)
    if twall is not None:
        prob.twall = twall
    conn = ot.TetConnectivity(mesh)
    fun = tm.sinusoids(prob.gamma, prob.mach, 3, 1e-3)
    prob.U, prob.Q, prob.UH, prob.Ustar = tm.packed_state(mesh, fun, conn.nfp, prob.ubc, seed)
    prob.Ustar = prob.Ustar + 1e-3 * np.sin(np.arange(prob.U.size))
    h = H.hdg_create_tet(mesh.vert_xyz, mesh.elem_vert, mesh.periodic_map, mesh.bnd_tag, mesh.elem_p, mesh.geo,
                         prob.gamma, prob.re, prob.pr, prob.mach)
    H.hdg_set_params(h, tau=prob.tau)
    if np.any(mesh.bnd_tag == 1):
        H.hdg_set_bc_state(h, 1, prob.ubc)
    if np.any(mesh.bnd_tag == 3):
        H.hdg_set_bc_state(h, 3, np.array([prob.twall]))
    dev = {k: torch.tensor(getattr(prob, k), dtype=torch.float64, device="cuda") for k in ("U", "Q", "UH", "Ustar")}
    return prob, ot.TetProblem(prob), h, dev


def block_errors(H, h, pb, vals_gpu):
    L = H.hdg_tet_layout(h)
    c = pb.conn
    vals, cache = pb.assemble()
    norms = [np.linalg.norm(vals[b]) for b in range(len(c.col))]
    scale = np.mean(norms)
    errs = []
    for b in range(len(c.col)):
        F = int(np.searchsorted(c.rowptr, b, side="right") - 1)
        bsF = c.hoff[F + 1] - c.hoff[F]
        bsG = c.hoff[c.col[b] + 1] - c.hoff[c.col[b]]
        got = vals_gpu[L["boff"][b]:L["boff"][b + 1]].reshape(bsG, bsF).T
        errs.append(np.linalg.norm(got - vals[b]) / max(norms[b], 1e-3 * scale))
    return np.array(errs), vals, cache


@pytest.mark.parametrize("k", [0, 1, 2])
def test_tet_linearize_condense_parity(H, k):
    mesh = mesh_case(k)
    prob, pb, h, dev = setup(H, mesh, twall=0.8 if k == 2 else None)
    try:
        s = H.hdg_tet_query(h)
        H.hdg_linearize_condense(h, dev["U"], dev["Q"], dev["UH"], dev["Ustar"], None, prob.dt, prob.a_ii)
        assert H.hdg_status(h) == H.HDG_OK
        vals = torch.zeros(s["n_vals"], dtype=torch.float64, device="cuda")
        H.hdg_get_blocks(h, vals)
        g = torch.zeros(s["n_trace"], dtype=torch.float64, device="cuda")
        H.hdg_trace_rhs(h, g)
        torch.cuda.synchronize()
        errs, ovals, cache = block_errors(H, h, pb, vals.cpu().numpy())
        assert errs.max() < TOL, errs.max()
        og = pb.assemble_g(cache)
        assert np.linalg.norm(g.cpu().numpy() - og) < TOL * np.linalg.norm(og)
        # trace matvec
        x = np.sin(0.37 * np.arange(s["n_trace"]))
        y = torch.zeros_like(g)
        H.hdg_trace_matvec(h, torch.tensor(x, device="cuda"), y)
        oy = pb.matvec(ovals, x)
        assert np.linalg.norm(y.cpu().numpy() - oy) < TOL * np.linalg.norm(oy)
        # recovery
        dUH = np.cos(0.11 * np.arange(s["n_trace"]))
        dQ = torch.zeros(3 * s["n_u"], dtype=torch.float64, device="cuda")
        dU = torch.zeros(s["n_u"], dtype=torch.float64, device="cuda")
        H.hdg_recover_interior(h, torch.tensor(dUH, device="cuda"), dQ, dU)
        dQc, dUc = dQ.cpu().numpy(), dU.cpu().numpy()
        c = pb.conn
        for e in range(mesh.n_elem):
            oq, ou = pb.recover(e, cache[e], dUH)
            ref = np.concatenate([oq.ravel(), ou.ravel()])
            got = np.concatenate([dQc[c.qoff[e]:c.qoff[e + 1]], dUc[c.uoff[e]:c.uoff[e + 1]]])
            assert np.linalg.norm(got - ref) < TOL * np.linalg.norm(ref), e
    finally:
        H.hdg_destroy(h)


def test_tet_freestream_gives_zero_rhs(H):
    """Uniform freestream with Q = 0 on the curved mixed mesh with far-field faces
    (a steady state there; next to a no-slip wall it is not): g = 0 to rounding."""
    mesh = mesh_case(0)
    prob, pb, h, dev = setup(H, mesh)
    try:
        s = H.hdg_tet_query(h)
        ub = torch.tensor(prob.ubc, device="cuda")
        L = H.hdg_tet_layout(h)
        U = torch.cat([ub.repeat_interleave(int((L["uoff"][e + 1] - L["uoff"][e]) // 5)) for e in range(mesh.n_elem)])
        UH = torch.cat([ub.repeat_interleave(int((L["hoff"][F + 1] - L["hoff"][F]) // 5))
                        for F in range(s["n_faces"])])
        Q = torch.zeros(3 * s["n_u"], dtype=torch.float64, device="cuda")
        H.hdg_linearize_condense(h, U, Q, UH, U.clone(), None, prob.dt, prob.a_ii)
        g = torch.zeros(s["n_trace"], dtype=torch.float64, device="cuda")
        H.hdg_trace_rhs(h, g)
        assert H.hdg_status(h) == H.HDG_OK
        assert g.abs().max().item() < 1e-12
    finally:
        H.hdg_destroy(h)
