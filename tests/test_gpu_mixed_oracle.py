"""Mixed-precision form against the FP64 oracle directly (GPU).

The mixed form's condensed blocks are an inexact linearization (FP32 Jacobian
terms, blocks and Schur product; FP64 interior LU and residual).  Their error
is measured against the oracle's FP64 blocks and right-hand side, block by
block, and bounded by the FP32 rounding level times the blocks' conditioning;
the Newton iteration, whose residual is evaluated in FP64, must reach the
oracle's own converged stage state (dense condensed Newton in FP64).
"""
import functools

import numpy as np
import pytest

import synth
from oracle.dirk import newton
from oracle.hdg import Problem
from tests.helpers import GpuRun, block_rel_errors

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_27863_gb300 import build
    build.build()


def mixed_blocks(run):
    from paper_2608_27863_gb300 import hdg as H
    s = run.sizes
    v = torch.empty(s["nnzb"] * s["block"] ** 2, dtype=torch.float32, device="cuda")
    H.hdg_get_blocks(run.h, v)
    torch.cuda.synchronize()
    return v.double().cpu().numpy().reshape(s["nnzb"], s["block"], s["block"]).transpose(0, 2, 1)


@pytest.mark.parametrize("make,rows,prec", [
    (synth.config1, None, "mixed"),
    (lambda: synth.config2(n=3), None, "3xtf32"),
    (lambda: synth.config3(n=3), [0, 17, 40, 63], "3xtf32"),
    (lambda: synth.tiny(3, 1, periodic=(True, False, True), visc_law=1, av=1e-3), None, "mixed"),
], ids=["quad-p2-fp32", "hex-p2-3xtf32", "hex-p3-av-3xtf32-sampled", "hex-p1-dirichlet-av-fp32"])
def test_mixed_blocks_and_rhs_against_oracle(make, rows, prec, record_property):
    from paper_2608_27863_gb300 import hdg as H
    P = make()
    run = GpuRun(P)
    mode = {"mixed": H.HDG_PREC_MIXED, "3xtf32": H.HDG_PREC_MIXED_3XTF32}[prec]
    H.hdg_set_params(run.h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s, precision=mode)
    run.linearize()
    assert H.hdg_status(run.h) == 0
    vals, g = mixed_blocks(run), run.rhs()
    pb = Problem(P)
    cn = pb.conn
    rows = range(cn.n_faces) if rows is None else rows
    blocks = [b for F in rows for b in range(cn.rowptr[F], cn.rowptr[F + 1])]
    orc, cache = pb.assemble(blocks=blocks)
    errs = block_rel_errors(vals, orc)
    og = pb.assemble_g(cache, rows)
    gerr = max(np.linalg.norm(g[F] - og[F]) / np.linalg.norm(og[F]) for F in rows)
    record_property("max_block_rel_err_vs_oracle", float(max(errs.values())))
    record_property("max_rhs_row_rel_err_vs_oracle", float(gerr))
    assert max(errs.values()) < 1e-3, max(errs.values())
    assert gerr < 1e-3, gerr
    run.close()


def test_mixed_tet_blocks_against_oracle(record_property):
    from paper_2608_27863_gb300 import hdg as H
    from tests.test_gpu_tet import block_errors, mesh_case, setup
    for k in (0, 1):
        prob, pb, h, dev = setup(H, mesh_case(k))
        try:
            H.hdg_set_params(h, tau=prob.tau, precision=H.HDG_PREC_MIXED)
            s = H.hdg_tet_query(h)
            H.hdg_linearize_condense(h, dev["U"], dev["Q"], dev["UH"], dev["Ustar"], None, prob.dt, prob.a_ii)
            assert H.hdg_status(h) == H.HDG_OK
            vals = torch.zeros(s["n_vals"], dtype=torch.float32, device="cuda")
            H.hdg_get_blocks(h, vals)
            g = torch.zeros(s["n_trace"], dtype=torch.float64, device="cuda")
            H.hdg_trace_rhs(h, g)
            errs, _, cache = block_errors(H, h, pb, vals.double().cpu().numpy())
            og = pb.assemble_g(cache)
            gerr = np.linalg.norm(g.cpu().numpy() - og) / np.linalg.norm(og)
            record_property("tet_case%d_max_block_rel_err_vs_oracle" % k, float(errs.max()))
            record_property("tet_case%d_rhs_rel_err_vs_oracle" % k, float(gerr))
            assert errs.max() < 1e-4, errs.max()
            assert gerr < 1e-4, gerr
        finally:
            H.hdg_destroy(h)


@functools.lru_cache(maxsize=1)
def oracle_root():
    P = synth.tiny(3, 2, seed=3)
    pb = Problem(P)
    oQ, oU, oUH, ohist = newton(pb, P.Q, P.U, P.UH, tol=1e-11, maxit=8)
    assert ohist[-1] <= 1e-11
    return oQ, oU, oUH


@pytest.mark.parametrize("prec", ["mixed", "3xtf32"])
def test_mixed_newton_reaches_oracle_state(prec, record_property):
    """Newton with the mixed linearization converges (FP64 residual) to the root the
    oracle's FP64 Newton finds."""
    from paper_2608_27863_gb300 import hdg as H
    P = synth.tiny(3, 2, seed=3)
    oQ, oU, oUH = oracle_root()
    run = GpuRun(P)
    mode = {"mixed": H.HDG_PREC_MIXED, "3xtf32": H.HDG_PREC_MIXED_3XTF32}[prec]
    H.hdg_set_params(run.h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s, precision=mode)
    nit, git, hist = H.hdg_newton(run.h, run.U, run.Q, run.UH, run.Ustar, run.nu, P.dt, P.a_ii, tol=1e-11,
                                  max_newton=30, restart=40, max_gmres=800, gmres_rtol=1e-12)
    assert hist[-1] <= 1e-11
    du = np.linalg.norm(run.U.cpu().numpy() - oU) / np.linalg.norm(oU)
    duh = np.linalg.norm(run.UH.cpu().numpy() - oUH) / np.linalg.norm(oUH)
    dq = np.linalg.norm(run.Q.cpu().numpy() - oQ) / np.linalg.norm(oQ)
    record_property("newton_iters", nit)
    record_property("state_rel_err_vs_oracle", [float(du), float(duh), float(dq)])
    assert du < 1e-10 and duh < 1e-10 and dq < 1e-9
    run.close()
