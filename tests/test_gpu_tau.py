"""State-dependent stabilization tau(uhat) = |vhat.n| + chat + mu / h on the GPU:
FP64 parity with the oracle (hex and tet, blocks, right-hand side, recovery
within 1e-11) and Newton with the mixed linearization."""
import numpy as np
import pytest

import synth
from oracle import tet as ot
from tests.helpers import GpuRun
from tests.test_gpu_parity import compare
from tests.test_gpu_tet import block_errors, mesh_case, setup

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,p,periodic", [(2, 2, True), (3, 1, False), (3, 2, True)])
def test_hex_state_dependent_tau_parity(dim, p, periodic):
    P = synth.tiny(dim, p, seed=11, periodic=periodic)
    P.tau_mode = 1
    assert compare(P, check_matvec=True) < 1e-11


def test_hex_state_dependent_tau_mixed_newton():
    from paper_2608_27863_gb300 import hdg as H
    P = synth.tiny(3, 2, seed=4)
    P.tau_mode = 1
    run = GpuRun(P)
    try:
        H.hdg_set_params(run.h, tau=P.tau, precision=H.HDG_PREC_MIXED, tau_mode=1)
        U, Q, UH = run.U.clone(), run.Q.clone(), run.UH.clone()
        nit, git, hist = H.hdg_newton(run.h, U, Q, UH, run.Ustar, None, P.dt, P.a_ii, tol=1e-10, max_newton=10,
                                      restart=60, max_gmres=600, gmres_rtol=1e-10)
        assert hist[-1] <= 1e-10
    finally:
        run.close()


def test_tet_state_dependent_tau_parity():
    from paper_2608_27863_gb300 import hdg as H
    mesh = mesh_case(1)
    prob, pb, h, dev = setup(H, mesh)
    try:
        prob.tau_mode = 1
        pb = ot.TetProblem(prob)
        H.hdg_set_params(h, tau=prob.tau, tau_mode=1)
        s = H.hdg_tet_query(h)
        H.hdg_linearize_condense(h, dev["U"], dev["Q"], dev["UH"], dev["Ustar"], None, prob.dt, prob.a_ii)
        assert H.hdg_status(h) == H.HDG_OK
        vals = torch.zeros(s["n_vals"], dtype=torch.float64, device="cuda")
        H.hdg_get_blocks(h, vals)
        g = torch.zeros(s["n_trace"], dtype=torch.float64, device="cuda")
        H.hdg_trace_rhs(h, g)
        errs, _, cache = block_errors(H, h, pb, vals.cpu().numpy())
        assert errs.max() < 1e-11, errs.max()
        og = pb.assemble_g(cache)
        assert np.linalg.norm(g.cpu().numpy() - og) < 1e-11 * np.linalg.norm(og)
        Rq = torch.zeros(3 * s["n_u"], dtype=torch.float64, device="cuda")
        Ru = torch.zeros(s["n_u"], dtype=torch.float64, device="cuda")
        Rh = torch.zeros(s["n_trace"], dtype=torch.float64, device="cuda")
        H.hdg_residual(h, dev["U"], dev["Q"], dev["UH"], dev["Ustar"], None, prob.dt, prob.a_ii, Rq, Ru, Rh)
        oq, ou, oh = pb.global_residual(pb.Q, pb.U, pb.UH)
        scale = np.linalg.norm(pb.U) + np.linalg.norm(pb.UH)
        for got, ref in ((Ru, ou), (Rh, oh)):
            assert np.linalg.norm(got.cpu().numpy() - ref) < 1e-12 * max(np.linalg.norm(ref), 1e-2 * scale)
    finally:
        H.hdg_destroy(h)
