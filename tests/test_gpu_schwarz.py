"""GPU additive Schwarz preconditioner (eq. additive-schwarz) vs the oracle.

The FP64 form must match the oracle's dense M_AS^{-1} x to 1e-10 relative;
the mixed form (FP32 patch factors) to 1e-4.  GMRES preconditioned with it
converges in fewer iterations than with block-Jacobi and reaches the dense
solution; Newton with it reaches the oracle's converged state.
"""
import numpy as np
import pytest

import synth
from oracle.dirk import dense_trace_matrix, newton
from oracle.hdg import Problem
from oracle.precond import additive_schwarz_matrix
from tests.helpers import GpuRun

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_27863_gb300 import build
    build.build()


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


CASES = {
    "quad-p2": synth.config1,
    "hex-p2": lambda: synth.config2(n=3),
    "quad-p3-dirichlet": lambda: synth.tiny(2, 3, periodic=(True, False), visc_law=1, av=1e-3),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_schwarz_apply_matches_oracle(name, prec):
    import torch
    from paper_2608_27863_gb300 import hdg as H
    P = CASES[name]()
    run = GpuRun(P)
    if prec == "mixed":
        H.hdg_set_params(run.h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s,
                         precision=H.HDG_PREC_MIXED)
    run.linearize()
    H.hdg_schwarz_setup(run.h)
    assert H.hdg_status(run.h) == 0
    c = H.hdg_get_connectivity(run.h)
    bs = run.sizes["block"]
    if prec == "fp64":
        S = dense_trace_matrix(run.blocks(), c["rowptr"], c["col"], bs)
    else:
        s = run.sizes
        v = torch.empty(s["nnzb"] * bs * bs, dtype=torch.float32, device="cuda")
        H.hdg_get_blocks(run.h, v)
        vals = v.cpu().numpy().astype(np.float64).reshape(s["nnzb"], bs, bs).transpose(0, 2, 1)
        S = dense_trace_matrix(vals, c["rowptr"], c["col"], bs)
    conn = Problem(P).conn
    Minv = additive_schwarz_matrix(S, conn, bs)
    rng = np.random.default_rng(5)
    for _ in range(2):
        x = rng.normal(size=P.UH.shape)
        xd = torch.from_numpy(x).cuda()
        y = torch.empty_like(xd)
        H.hdg_schwarz_apply(run.h, xd, y)
        torch.cuda.synchronize()
        ref = Minv @ x.ravel()
        assert rel(y.cpu().numpy(), ref) < (1e-10 if prec == "fp64" else 1e-4)
    # bitwise reproducible
    y2 = torch.empty_like(xd)
    H.hdg_schwarz_apply(run.h, xd, y2)
    assert torch.equal(y, y2)
    run.close()


def test_gmres_with_schwarz_beats_block_jacobi():
    import torch
    from paper_2608_27863_gb300 import hdg as H
    P = synth.config2(n=3)
    run = GpuRun(P).linearize()
    g = torch.from_numpy(run.rhs()).cuda()
    H.hdg_blockjacobi_setup(run.h)
    x1 = torch.zeros_like(g)
    it_bj, r1 = H.hdg_gmres(run.h, g, x1, restart=60, max_iter=1000, rtol=1e-10, precond=True)
    H.hdg_set_preconditioner(run.h, H.HDG_PC_SCHWARZ)
    H.hdg_schwarz_setup(run.h)
    x2 = torch.zeros_like(g)
    it_as, r2 = H.hdg_gmres(run.h, g, x2, restart=60, max_iter=1000, rtol=1e-10, precond=True)
    assert it_as < it_bj, (it_as, it_bj)
    c = H.hdg_get_connectivity(run.h)
    S = dense_trace_matrix(run.blocks(), c["rowptr"], c["col"], run.sizes["block"])
    xd = np.linalg.solve(S, g.cpu().numpy().ravel())
    assert rel(x2.cpu().numpy(), xd) < 1e-7
    run.close()


def test_newton_with_schwarz_matches_oracle():
    from paper_2608_27863_gb300 import hdg as H
    P = synth.config1()
    run = GpuRun(P)
    H.hdg_set_preconditioner(run.h, H.HDG_PC_SCHWARZ)
    hist = H.hdg_newton_fixed(run.h, run.U, run.Q, run.UH, run.Ustar, run.nu, P.dt, P.a_ii,
                              n_newton=5, m=30, use_graph=True)
    assert hist[-1] <= 1e-10, hist
    pb = Problem(P)
    oq, ou, oh, _ = newton(pb, pb.Q, pb.U, pb.UH, tol=1e-12)
    assert rel(run.U.cpu().numpy(), ou) < 1e-10 and rel(run.UH.cpu().numpy(), oh) < 1e-10
    run.close()
