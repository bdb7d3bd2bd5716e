"""The wall-bounded workload (hypersonic flat-plate boundary layer, hex p = 3,
graded wall-normal cells, isothermal wall, far-field / inflow, outflow,
periodic span, Sutherland viscosity, artificial viscosity on).

* small meshes of the same construction: FP64 path vs the oracle, in full
  (p = 2) and on sampled rows (p = 3); the mixed form vs the FP64 form;
* the full 64 x 48 x 32 = 98,304-element mesh in the mixed form (the FP64
  arrays are never allocated): probed through the trace matvec against the
  oracle's blocks of sampled faces, and its device footprint.
"""
import numpy as np
import pytest

import synth
from oracle.av import av_field
from oracle.hdg import Problem
from oracle.refelem import RefElem
from tests.helpers import GpuRun
from tests.test_gpu_parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_27863_gb300 import build
    build.build()


def with_av(P, c_av=2e-3):
    """The lagged AV field of the state (oracle sensor + smoothing), as an input."""
    h_m = 0.1 / P.mesh.n[1]
    P.nu = av_field(P, P.U, P.Q, c_av, h_m, 1.0, RefElem(3, P.p).nodes1)
    return P


def test_plate_p2_full():
    P = with_av(synth.config5(4, 6, 3, 2))
    assert P.nu.max() > 0
    compare(P, check_matvec=True)


def test_plate_p3_sampled():
    P = with_av(synth.config5(3, 5, 3, 3))
    compare(P, rows=[0, 7, 31, 58])


def test_plate_mixed_against_fp64():
    import torch
    from paper_2608_27863_gb300 import hdg as H
    P = with_av(synth.config5(4, 6, 3, 2))
    run = GpuRun(P).linearize()
    v64 = run.blocks()
    H.hdg_set_params(run.h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s,
                     precision=H.HDG_PREC_MIXED_3XTF32)
    run.linearize()
    assert H.hdg_status(run.h) == 0
    s = run.sizes
    v = torch.empty(s["nnzb"] * s["block"] ** 2, dtype=torch.float32, device="cuda")
    H.hdg_get_blocks(run.h, v)
    v32 = v.cpu().numpy().astype(np.float64).reshape(s["nnzb"], s["block"], s["block"]).transpose(0, 2, 1)
    err = np.linalg.norm(v32 - v64) / np.linalg.norm(v64)
    assert err < 1e-4, err
    # Newton in the mixed form reaches the FP64 residual tolerance
    nit, git, hist = H.hdg_newton(run.h, run.U, run.Q, run.UH, run.Ustar, run.nu, P.dt, P.a_ii, tol=1e-8,
                                  max_newton=10, restart=60, max_gmres=800, gmres_rtol=1e-10)
    assert hist[-1] <= 1e-8, hist
    run.close()


def test_plate_full_size_mixed():
    import torch
    from paper_2608_27863_gb300 import hdg as H
    P = synth.config5()
    assert P.mesh.n_elem == 98304
    run = GpuRun(P)
    nu = torch.empty_like(run.U[:, 0, :]).contiguous()
    H.hdg_av_field(run.h, run.U, run.Q, nu, 2e-3, 0.1 / 48, 1.0)
    run.nu = nu
    H.hdg_set_params(run.h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s,
                     precision=H.HDG_PREC_MIXED_3XTF32)
    run.linearize()
    assert H.hdg_status(run.h) == 0
    sizes = H.hdg_query_sizes(run.h)
    assert sizes["device_bytes"] < 250e9, sizes["device_bytes"]
    c = H.hdg_get_connectivity(run.h)
    bs = sizes["block"]
    Pn = P
    Pn.nu = nu.cpu().numpy()
    pb = Problem(Pn)
    rng = np.random.default_rng(0)
    faces = [int(f) for f in synth.splitmix64(31, 2) % np.uint64(sizes["n_faces"])]
    for G in faces:
        x = np.zeros((sizes["n_faces"], bs))
        x[G] = rng.normal(size=bs)
        y = run.matvec(x.reshape(P.UH.shape)).reshape(sizes["n_faces"], bs)
        # rows coupled to G: the faces of the elements on G
        elems = [e for e in c["f2e"][G] if e >= 0]
        rows = sorted({int(F) for e in elems for F in c["e2f"][e]})
        blocks = []
        for F in rows:
            for b in range(c["rowptr"][F], c["rowptr"][F + 1]):
                if c["col"][b] == G:
                    blocks.append(b)
        orc, _ = pb.assemble(blocks=blocks)
        for F, b in zip(rows, blocks):
            ref = orc[b] @ x[G]
            assert np.linalg.norm(y[F] - ref) <= 1e-3 * np.linalg.norm(ref) + 1e-6 * np.linalg.norm(x[G]), (G, F)
    run.close()
