"""Additive Schwarz on tetrahedral handles (Sec. 3.3, eq. additive-schwarz), GPU.

Patches of element faces of mixed degree (t = 60 .. 300 unknowns):
* y = M^{-1} x against the oracle's dense M_AS^{-1} = sum_r R_r^T S_r^{-1} R_r
  of the same assembled operator: 1e-10 relative for FP64 factors, 1e-4 for
  the mixed form's FP32 factors;
* GMRES preconditioned with it needs fewer iterations than with block-Jacobi
  and reaches the dense solution;
* Newton with it reaches the oracle's converged stage state.
"""
import numpy as np
import pytest

from oracle import tet as ot
from oracle.precond import additive_schwarz_matrix_offsets

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_27863_gb300 import build
    build.build()
    from paper_2608_27863_gb300 import hdg
    return hdg


def dense_operator(H, h, vals):
    """The assembled trace operator as a dense matrix (block b of row F, column G at
    boff[b], bs_F x bs_G column-major)."""
    L = H.hdg_tet_layout(h)
    hoff, boff, rowptr, col = L["hoff"], L["boff"], L["rowptr"], L["col"]
    n = int(hoff[-1])
    S = np.zeros((n, n))
    for F in range(len(hoff) - 1):
        for b in range(rowptr[F], rowptr[F + 1]):
            G = col[b]
            bF, bG = hoff[F + 1] - hoff[F], hoff[G + 1] - hoff[G]
            S[hoff[F]:hoff[F + 1], hoff[G]:hoff[G + 1]] = vals[boff[b]:boff[b + 1]].reshape(bG, bF).T
    return S, L


def linearized(H, k, prec):
    from tests.test_gpu_tet import mesh_case, setup
    prob, pb, h, dev = setup(H, mesh_case(k))
    H.hdg_set_params(h, tau=prob.tau, precision=H.HDG_PREC_FP64 if prec == "fp64" else H.HDG_PREC_MIXED)
    H.hdg_linearize_condense(h, dev["U"], dev["Q"], dev["UH"], dev["Ustar"], None, prob.dt, prob.a_ii)
    return prob, pb, h, dev


@pytest.mark.parametrize("k", [0, 1])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_tet_schwarz_apply_matches_oracle(H, k, prec):
    prob, pb, h, dev = linearized(H, k, prec)
    try:
        s = H.hdg_tet_query(h)
        H.hdg_schwarz_setup(h)
        assert H.hdg_status(h) == H.HDG_OK
        vals = torch.zeros(s["n_vals"], dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")
        H.hdg_get_blocks(h, vals)
        S, L = dense_operator(H, h, vals.double().cpu().numpy())
        M = additive_schwarz_matrix_offsets(S, L["e2f"], L["hoff"])
        x = torch.from_numpy(np.random.default_rng(k).normal(size=s["n_trace"])).cuda()
        y = torch.empty_like(x)
        H.hdg_schwarz_apply(h, x, y)
        ref = M @ x.cpu().numpy()
        err = np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err < (1e-10 if prec == "fp64" else 1e-4), err
        y2 = torch.empty_like(x)
        H.hdg_schwarz_apply(h, x, y2)
        assert torch.equal(y, y2)                       # fixed summation order
    finally:
        H.hdg_destroy(h)


def test_tet_gmres_schwarz_fewer_iterations(H, record_property):
    prob, pb, h, dev = linearized(H, 1, "fp64")
    try:
        s = H.hdg_tet_query(h)
        g = torch.zeros(s["n_trace"], dtype=torch.float64, device="cuda")
        H.hdg_trace_rhs(h, g)
        vals = torch.zeros(s["n_vals"], dtype=torch.float64, device="cuda")
        H.hdg_get_blocks(h, vals)
        S, _ = dense_operator(H, h, vals.cpu().numpy())
        xref = np.linalg.solve(S, g.cpu().numpy())
        its = {}
        for name, kind in (("bj", H.HDG_PC_BLOCKJACOBI), ("schwarz", H.HDG_PC_SCHWARZ)):
            H.hdg_set_preconditioner(h, kind)
            if kind == H.HDG_PC_SCHWARZ:
                H.hdg_schwarz_setup(h)
            else:
                H.hdg_blockjacobi_setup(h)
            x = torch.zeros_like(g)
            it, rel = H.hdg_gmres(h, g, x, restart=200, max_iter=400, rtol=1e-10, precond=True)
            its[name] = it
            assert np.linalg.norm(x.cpu().numpy() - xref) < 1e-8 * np.linalg.norm(xref)
        record_property("gmres_iterations", its)
        assert its["schwarz"] < its["bj"], its
    finally:
        H.hdg_destroy(h)


def test_tet_newton_schwarz_reaches_oracle_state(H):
    from tests.test_gpu_tet import mesh_case, setup
    prob, pb, h, dev = setup(H, mesh_case(0))
    try:
        H.hdg_set_preconditioner(h, H.HDG_PC_SCHWARZ)
        U, Q, UH = dev["U"].clone(), dev["Q"].clone(), dev["UH"].clone()
        nit, git, hist = H.hdg_newton(h, U, Q, UH, dev["Ustar"], None, prob.dt, prob.a_ii, tol=1e-10,
                                      max_newton=8, restart=60, max_gmres=600, gmres_rtol=1e-12)
        assert hist[-1] <= 1e-10
        oQ, oU, oUH, ohist = ot.newton(pb, pb.Q, pb.U, pb.UH, tol=1e-11, maxit=8)
        assert np.linalg.norm(U.cpu().numpy() - oU) < 1e-9 * np.linalg.norm(oU)
        assert np.linalg.norm(UH.cpu().numpy() - oUH) < 1e-9 * np.linalg.norm(oUH)
    finally:
        H.hdg_destroy(h)
