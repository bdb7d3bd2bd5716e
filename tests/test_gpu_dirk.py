"""GPU Newton with fixed-length GMRES, its CUDA-graph replay, and the DIRK step.

* hdg_newton_fixed reaches the oracle's converged Newton state, and the
  graph replay gives bitwise the same result as the eager launches;
* hdg_dirk_step (Alexander's SDIRK3, every stage and Newton iteration in one
  CUDA graph) matches the oracle's DIRK step, on a periodic mesh and on one
  with Dirichlet faces, and conserves the integrals on the periodic mesh.
"""
import numpy as np
import pytest

import synth
from oracle.dirk import alexander_sdirk3, hdg_dirk_step, newton
from oracle.hdg import Problem
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


def host(run):
    return run.Q.cpu().numpy(), run.U.cpu().numpy(), run.UH.cpu().numpy()


def test_newton_fixed_matches_oracle_and_graph_is_bitwise():
    from paper_2608_27863_gb300 import hdg as H
    P = synth.config1()
    eager, graph = GpuRun(P), GpuRun(P)
    h1 = H.hdg_newton_fixed(eager.h, eager.U, eager.Q, eager.UH, eager.Ustar, eager.nu, P.dt, P.a_ii,
                            n_newton=6, m=60, use_graph=False)
    h2 = H.hdg_newton_fixed(graph.h, graph.U, graph.Q, graph.UH, graph.Ustar, graph.nu, P.dt, P.a_ii,
                            n_newton=6, m=60, use_graph=True)
    assert np.array_equal(h1, h2)
    for a, b in zip(host(eager), host(graph)):
        assert np.array_equal(a, b)
    assert h1[-1] <= 1e-10, h1
    pb = Problem(P)
    oq, ou, oh, ohist = newton(pb, pb.Q, pb.U, pb.UH, tol=1e-12)
    assert abs(h1[0] - ohist[0]) <= 1e-11 * ohist[0]
    q, u, uh = host(graph)
    assert rel(u, ou) < 1e-10 and rel(uh, oh) < 1e-10 and rel(q, oq) < 1e-8
    # a second call replays the same graph from the converged state
    h3 = H.hdg_newton_fixed(graph.h, graph.U, graph.Q, graph.UH, graph.Ustar, graph.nu, P.dt, P.a_ii,
                            n_newton=6, m=60, use_graph=True)
    assert h3[-1] <= 1e-10
    eager.close()
    graph.close()


def test_newton_fixed_mixed_precision():
    from paper_2608_27863_gb300 import hdg as H
    P = synth.config2(n=3)
    run = GpuRun(P)
    H.hdg_set_params(run.h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s,
                     precision=H.HDG_PREC_MIXED_3XTF32)
    hist = H.hdg_newton_fixed(run.h, run.U, run.Q, run.UH, run.Ustar, run.nu, P.dt, P.a_ii,
                              n_newton=6, m=40, use_graph=True)
    assert hist[-1] <= 1e-8 * hist[0], hist
    run.close()


def gpu_dirk(P, n_newton, m, use_graph):
    from paper_2608_27863_gb300 import hdg as H
    run = GpuRun(P)
    A, b = H.sdirk3_tableau()
    hist = H.hdg_dirk_step(run.h, run.U, run.Q, run.UH, run.nu, P.dt, A, b, n_newton=n_newton, m=m,
                           use_graph=use_graph)
    out = host(run)
    run.close()
    return out, hist


@pytest.mark.parametrize("per", [True, (True, False)], ids=["periodic", "dirichlet"])
def test_dirk_step_matches_oracle(per):
    from paper_2608_27863_gb300 import hdg as H
    A, b = H.sdirk3_tableau()
    Ao, bo, _ = alexander_sdirk3()
    assert np.abs(A - Ao).max() < 1e-14 and np.abs(b - bo).max() < 1e-14
    P = synth.tiny(2, 2, seed=3, periodic=per)
    P.Ustar = P.U.copy()
    (q, u, uh), hist = gpu_dirk(P, n_newton=5, m=60, use_graph=True)
    (q2, u2, uh2), hist2 = gpu_dirk(P, n_newton=5, m=60, use_graph=False)
    assert np.array_equal(u, u2) and np.array_equal(uh, uh2) and np.array_equal(hist, hist2)
    assert np.all(hist[:, -1] <= 1e-10), hist
    oq, ou, oh, ohists = hdg_dirk_step(P, Ao, bo, tol=1e-12)
    assert rel(u, ou) < 1e-10 and rel(uh, oh) < 1e-10 and rel(q, oq) < 1e-8
    for s in range(3):                       # the stage's first residual matches the oracle's
        assert abs(hist[s, 0] - ohists[s][0]) <= 1e-9 * ohists[s][0]
    if per is True:
        pb = Problem(P)
        w = np.stack([pb.geom(e).M.sum(axis=1) for e in range(P.mesh.n_elem)])
        before = np.einsum("ei,eai->a", w, P.U)
        after = np.einsum("ei,eai->a", w, u)
        assert np.abs(after - before).max() < 1e-11 * np.abs(before).max()


def test_dirk_rejects_bad_tableaus():
    import torch
    from paper_2608_27863_gb300 import hdg as H
    P = synth.tiny(2, 1)
    run = GpuRun(P)
    g = (3 + np.sqrt(3)) / 6
    with pytest.raises(H.HDGError) as ex:      # not stiffly accurate
        H.hdg_dirk_step(run.h, run.U, run.Q, run.UH, run.nu, P.dt, np.array([[g, 0], [1 - 2 * g, g]]),
                        np.array([0.5, 0.5]))
    assert ex.value.code == H.HDG_EUNSUPPORTED
    with pytest.raises(H.HDGError) as ex:      # not lower triangular
        H.hdg_dirk_step(run.h, run.U, run.Q, run.UH, run.nu, P.dt, np.array([[0.5, 0.1], [0.5, 0.5]]),
                        np.array([0.5, 0.5]))
    assert ex.value.code == H.HDG_EINVAL
    u0 = P.U
    assert np.array_equal(run.U.cpu().numpy(), u0)   # nothing ran
    run.close()
