"""GPU consumer loop (FP64): stage residual, block-Jacobi, GMRES and Newton.

The residual is compared with the oracle's global residual vector by vector;
GMRES against a dense solve of the same assembled operator; the Newton
iteration against the oracle's own Newton iteration (dense condensed solve +
recovery per step), which must reach the same converged stage state.
"""
import numpy as np
import pytest

import synth
from oracle.hdg import Problem
from tests.helpers import GpuRun

pytestmark = pytest.mark.gpu
TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_27863_gb300 import build
    build.build()


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.mark.parametrize("make", [synth.config1, lambda: synth.config2(n=3), lambda: synth.config3(n=3),
                                  lambda: synth.tiny(2, 3, visc_law=1, av=2e-3),
                                  lambda: synth.tiny(3, 1, periodic=(True, False, True))],
                         ids=["quad-p2", "hex-p2", "hex-p3-av", "quad-p3-av", "hex-p1-dirichlet"])
def test_residual_matches_oracle(make):
    import torch
    from paper_2608_27863_gb300 import hdg as H
    P = make()
    run = GpuRun(P)
    Rq, Ru, Ruh = torch.empty_like(run.Q), torch.empty_like(run.U), torch.empty_like(run.UH)
    norms = H.hdg_residual(run.h, run.U, run.Q, run.UH, run.Ustar, run.nu, P.dt, P.a_ii, Rq, Ru, Ruh)
    pb = Problem(P)
    oq, ou, oh = pb.global_residual(pb.Q, pb.U, pb.UH)
    assert rel(Rq.cpu().numpy(), oq) < TOL
    assert rel(Ru.cpu().numpy(), ou) < TOL
    assert rel(Ruh.cpu().numpy(), oh) < TOL
    full = np.sqrt(np.sum(oq ** 2) + np.sum(ou ** 2) + np.sum(oh ** 2))
    assert abs(norms[0] - full) < TOL * full
    assert abs(norms[2] - np.linalg.norm(oh)) < TOL * np.linalg.norm(oh)
    run.close()


def dense_from_blocks(vals, rowptr, col, bs):
    F = len(rowptr) - 1
    S = np.zeros((F * bs, F * bs))
    for f in range(F):
        for b in range(rowptr[f], rowptr[f + 1]):
            S[f * bs:(f + 1) * bs, col[b] * bs:(col[b] + 1) * bs] = vals[b]
    return S


@pytest.mark.parametrize("make", [synth.config1, lambda: synth.config2(n=3)], ids=["quad-p2", "hex-p2"])
def test_blockjacobi_and_gmres(make):
    import torch
    from paper_2608_27863_gb300 import hdg as H
    P = make()
    run = GpuRun(P).linearize()
    vals = run.blocks()
    c = H.hdg_get_connectivity(run.h)
    bs = run.sizes["block"]
    g = torch.from_numpy(run.rhs()).cuda()
    H.hdg_blockjacobi_setup(run.h)
    assert H.hdg_status(run.h) == 0
    # block-Jacobi inverts the diagonal blocks
    x = torch.randn_like(g)
    y = torch.empty_like(g)
    H.hdg_blockjacobi_apply(run.h, x, y)
    xv, yv = x.cpu().numpy().reshape(-1, bs), y.cpu().numpy().reshape(-1, bs)
    for f in range(len(c["rowptr"]) - 1):
        d = [b for b in range(c["rowptr"][f], c["rowptr"][f + 1]) if c["col"][b] == f][0]
        assert np.allclose(vals[d] @ yv[f], xv[f], rtol=1e-10, atol=1e-10 * np.abs(xv[f]).max())
    # GMRES against a dense solve of the same operator
    sol = torch.zeros_like(g)
    it, relres = H.hdg_gmres(run.h, g, sol, restart=40, max_iter=600, rtol=1e-12, precond=True)
    assert relres <= 1e-12 and it > 0
    Sd = dense_from_blocks(vals, c["rowptr"], c["col"], bs)
    gd = g.cpu().numpy().ravel()
    xd = np.linalg.solve(Sd, gd)
    xs = sol.cpu().numpy().ravel()
    assert np.linalg.norm(Sd @ xs - gd) <= 1e-9 * np.linalg.norm(gd)
    assert rel(xs, xd) < 1e-8
    # unpreconditioned path as well
    sol2 = torch.zeros_like(g)
    it2, rel2 = H.hdg_gmres(run.h, g, sol2, restart=60, max_iter=2000, rtol=1e-11, precond=False,
                            raise_on_noconv=False)
    assert np.linalg.norm(Sd @ sol2.cpu().numpy().ravel() - gd) <= 1e-8 * np.linalg.norm(gd)
    run.close()


def oracle_newton(P, tol, maxit=8):
    """Newton on the stage equations with the oracle's dense condensed solve."""
    pb = Problem(P)
    Q, U, UH = pb.Q.copy(), pb.U.copy(), pb.UH.copy()
    hist = []
    cn = pb.conn
    bs = pb.ref.m * pb.ref.Nfp
    for k in range(maxit + 1):
        hist.append(pb.residual_norm(Q, U, UH))
        if hist[-1] <= tol:
            break
        pb.Q, pb.U, pb.UH = Q, U, UH
        pb._geom = pb._geom
        vals, cache = pb.assemble()
        S = dense_from_blocks(vals, cn.rowptr, cn.col, bs)
        gg = pb.assemble_g(cache, range(cn.n_faces))
        g = np.concatenate([gg[f].ravel() for f in range(cn.n_faces)])
        dUH = np.linalg.solve(S, g).reshape(UH.shape)
        dQ = np.zeros_like(Q)
        dU = np.zeros_like(U)
        for e in range(P.mesh.n_elem):
            dQ[e], dU[e] = pb.recover(e, cache[e], dUH)
        Q, U, UH = Q + dQ, U + dU, UH + dUH
    return Q, U, UH, hist


def test_newton_matches_oracle_newton():
    from paper_2608_27863_gb300 import hdg as H
    P = synth.config1()
    run = GpuRun(P)
    nit, git, hist = H.hdg_newton(run.h, run.U, run.Q, run.UH, run.Ustar, run.nu, P.dt, P.a_ii, tol=1e-11,
                                  max_newton=8, restart=40, max_gmres=600, gmres_rtol=1e-12)
    assert hist[-1] <= 1e-11 and nit <= 6
    # quadratic convergence once in the asymptotic range
    assert hist[-1] < 1e-3 * hist[-2] or hist[-2] < 1e-8
    oq, ou, oh, ohist = oracle_newton(P, 1e-11)
    assert len(ohist) == len(hist)
    assert rel(run.U.cpu().numpy(), ou) < 1e-12
    assert rel(run.UH.cpu().numpy(), oh) < 1e-12
    assert rel(run.Q.cpu().numpy(), oq) < 1e-10
    run.close()


def test_newton_hex_p2_small():
    from paper_2608_27863_gb300 import hdg as H
    P = synth.config2(n=4)
    run = GpuRun(P)
    nit, git, hist = H.hdg_newton(run.h, run.U, run.Q, run.UH, run.Ustar, run.nu, P.dt, P.a_ii, tol=1e-9,
                                  max_newton=10, restart=40, max_gmres=800, gmres_rtol=1e-11)
    assert hist[-1] <= 1e-9
    assert all(hist[i + 1] < hist[i] for i in range(len(hist) - 1))
    run.close()


def test_newton_with_dirichlet_boundary_matches_oracle():
    from paper_2608_27863_gb300 import hdg as H
    P = synth.tiny(2, 2, periodic=(True, False))
    run = GpuRun(P)
    nit, git, hist = H.hdg_newton(run.h, run.U, run.Q, run.UH, run.Ustar, run.nu, P.dt, P.a_ii, tol=1e-11,
                                  max_newton=8, restart=40, max_gmres=600, gmres_rtol=1e-12)
    assert hist[-1] <= 1e-11
    oq, ou, oh, ohist = oracle_newton(P, 1e-11)
    assert rel(run.U.cpu().numpy(), ou) < 1e-11
    assert rel(run.UH.cpu().numpy(), oh) < 1e-11
    run.close()


@pytest.mark.parametrize("tags", [{(0, 0): 1, (0, 1): 2}, {(1, 0): 3, (1, 1): 4}], ids=["inflow-outflow", "walls"])
def test_residual_and_newton_with_walls(tags):
    import torch
    from paper_2608_27863_gb300 import hdg as H
    from tests.test_gpu_parity import tagged
    per = (False, True) if (0, 0) in tags else (True, False)
    P = tagged(synth.tiny(2, 2, periodic=per, visc_law=1, mach=0.4), tags, twall=1.1)
    run = GpuRun(P)
    Rq, Ru, Ruh = torch.empty_like(run.Q), torch.empty_like(run.U), torch.empty_like(run.UH)
    H.hdg_residual(run.h, run.U, run.Q, run.UH, run.Ustar, run.nu, P.dt, P.a_ii, Rq, Ru, Ruh)
    pb = Problem(P)
    oq, ou, oh = pb.global_residual(pb.Q, pb.U, pb.UH)
    assert rel(Ruh.cpu().numpy(), oh) < TOL and rel(Ru.cpu().numpy(), ou) < TOL
    nit, git, hist = H.hdg_newton(run.h, run.U, run.Q, run.UH, run.Ustar, run.nu, P.dt, P.a_ii, tol=1e-11,
                                  max_newton=10, restart=60, max_gmres=600, gmres_rtol=1e-12)
    assert hist[-1] <= 1e-11
    oq2, ou2, oh2, _ = oracle_newton(P, 1e-11, maxit=10)
    assert rel(run.U.cpu().numpy(), ou2) < 1e-10 and rel(run.UH.cpu().numpy(), oh2) < 1e-10
    run.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_linearize_returns_the_fp64_residual_norm(prec):
    """res_norm of hdg_linearize_condense: the FP64 ||F(W)||_2 at the linearization
    point, equal to the oracle's global residual norm whatever the system precision;
    the condensed system is the same as without it."""
    from paper_2608_27863_gb300 import hdg as H
    P = synth.tiny(3, 2, seed=5, periodic=(True, False, True))
    run = GpuRun(P)
    if prec == "mixed":
        H.hdg_set_params(run.h, tau=P.tau, precision=H.HDG_PREC_MIXED)
    H.hdg_linearize_condense(run.h, run.U, run.Q, run.UH, run.Ustar, run.nu, P.dt, P.a_ii)
    v0, g0 = run.blocks(), run.rhs()
    r = H.hdg_linearize_condense(run.h, run.U, run.Q, run.UH, run.Ustar, run.nu, P.dt, P.a_ii, res_norm=True)
    pb = Problem(P)
    oq, ou, oh = pb.global_residual(pb.Q, pb.U, pb.UH)
    full = np.sqrt(np.sum(oq ** 2) + np.sum(ou ** 2) + np.sum(oh ** 2))
    assert abs(r - full) < TOL * full
    assert np.array_equal(run.blocks(), v0) and np.array_equal(run.rhs(), g0)
    run.close()
