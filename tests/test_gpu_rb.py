"""GPU reduced-basis initial guess (eq. rb-min) vs the oracle.

* hdg_rb_guess matches the oracle's least-squares guess for the same window
  (columns pushed through hdg_rb_push, products S w taken with the GPU's own
  assembled operator), including the wrap-around of a full window;
* columns that solve S w_i = g_i reproduce the solution of any combination
  of the g_i;
* in a sequence of stage solves, Newton with the window reaches the same
  state as without it in no more GMRES iterations.
"""
import numpy as np
import pytest

import synth
from oracle.dirk import dense_trace_matrix
from oracle.rb import ReducedBasis
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


@pytest.mark.parametrize("nb_max,pushes", [(6, 4), (3, 5), (20, 20)])
def test_guess_matches_oracle(nb_max, pushes):
    import torch
    from paper_2608_27863_gb300 import hdg as H
    P = synth.config1()
    run = GpuRun(P).linearize()
    c = H.hdg_get_connectivity(run.h)
    S = dense_trace_matrix(run.blocks(), c["rowptr"], c["col"], run.sizes["block"])
    H.hdg_rb_setup(run.h, nb_max)
    orb = ReducedBasis(nb_max)
    rng = np.random.default_rng(nb_max + pushes)
    x0 = torch.empty_like(run.UH)
    g = torch.from_numpy(rng.normal(size=P.UH.shape)).cuda()
    H.hdg_rb_guess(run.h, g, x0)                      # empty window: zero guess
    assert torch.count_nonzero(x0) == 0
    for _ in range(pushes):
        w = rng.normal(size=P.UH.shape)
        H.hdg_rb_push(run.h, torch.from_numpy(w).cuda())
        orb.push(w, S @ w.ravel())
    for _ in range(2):
        gn = rng.normal(size=P.UH.shape)
        H.hdg_rb_guess(run.h, torch.from_numpy(gn).cuda(), x0)
        torch.cuda.synchronize()
        assert rel(x0.cpu().numpy(), orb.guess(gn)) < 1e-9
    run.close()


def test_previous_solutions_reproduce_combinations():
    import torch
    from paper_2608_27863_gb300 import hdg as H
    P = synth.config2(n=3)
    run = GpuRun(P).linearize()
    H.hdg_blockjacobi_setup(run.h)
    H.hdg_rb_setup(run.h, 4)
    rng = np.random.default_rng(3)
    G = [torch.from_numpy(rng.normal(size=P.UH.shape)).cuda() for _ in range(3)]
    X = []
    for gi in G:
        x = torch.zeros_like(gi)
        H.hdg_gmres(run.h, gi, x, restart=60, max_iter=600, rtol=1e-13, precond=True)
        H.hdg_rb_push(run.h, x)
        X.append(x)
    g = 0.5 * G[0] - 2.0 * G[1] + G[2]
    x0 = torch.empty_like(g)
    H.hdg_rb_guess(run.h, g, x0)
    xs = 0.5 * X[0] - 2.0 * X[1] + X[2]
    assert rel(x0.cpu().numpy(), xs.cpu().numpy()) < 1e-8
    # GMRES from that guess converges at once
    it, r = H.hdg_gmres(run.h, g, x0, restart=60, max_iter=600, rtol=1e-9, precond=True)
    assert it <= 1
    run.close()


def test_newton_sequence_with_reduced_basis():
    from paper_2608_27863_gb300 import hdg as H
    P = synth.config2(n=3)
    results = []
    for nb in (0, 8):
        run = GpuRun(P)
        H.hdg_rb_setup(run.h, nb)
        total = 0
        for stage in range(3):
            # a sequence of closely related stage problems: U* drifts slightly
            run.Ustar.mul_(1.0 + 1e-3 * (stage + 1))
            nit, git, hist = H.hdg_newton(run.h, run.U, run.Q, run.UH, run.Ustar, run.nu, P.dt, P.a_ii, tol=1e-9,
                                          max_newton=10, restart=60, max_gmres=600, gmres_rtol=1e-6)
            total += git
        results.append((total, run.U.cpu().numpy(), run.UH.cpu().numpy()))
        run.close()
    (t0, u0, h0), (t1, u1, h1) = results
    assert t1 <= t0, (t1, t0)
    assert rel(u1, u0) < 1e-8 and rel(h1, h0) < 1e-8
