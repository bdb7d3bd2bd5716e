"""Per-element Schur complements S^K (hdg_set_element_block_output) against the
oracle's condensation of the same element (GPU): FP64 within 1e-11 relative per
element (quad / hex with either Schur-product kernel, tetrahedra of mixed degree),
the mixed form's FP32 blocks within 1e-3."""
import numpy as np
import pytest

import synth
from oracle.hdg import Problem
from tests.helpers import GpuRun

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_27863_gb300 import build
    build.build()
    from paper_2608_27863_gb300 import hdg
    return hdg


@pytest.mark.parametrize("make,tuning,prec", [
    (lambda: synth.config2(n=3), dict(schur_mode=0), "fp64"),
    (lambda: synth.config2(n=3), dict(schur_mode=3), "fp64"),
    (lambda: synth.tiny(2, 3, periodic=(True, False), visc_law=1, av=1e-3), dict(schur_mode=0), "fp64"),
    (lambda: synth.config2(n=3), None, "mixed"),
], ids=["hex-p2", "hex-p2-tensor-core-schur", "quad-p3-dirichlet", "hex-p2-mixed"])
def test_element_blocks_match_oracle(H, make, tuning, prec):
    P = make()
    run = GpuRun(P)
    if prec == "mixed":
        H.hdg_set_params(run.h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s,
                         precision=H.HDG_PREC_MIXED)
    if tuning:
        H.hdg_set_tuning(run.h, **tuning)
    t = run.sizes["t"]
    E = run.sizes["n_elem"]
    SK = torch.zeros(E * t * t, dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")
    H.hdg_set_element_block_output(run.h, SK)
    run.linearize()
    assert H.hdg_status(run.h) == 0
    got = SK.double().cpu().numpy().reshape(E, t, t)
    pb = Problem(P)
    tol = 1e-11 if prec == "fp64" else 1e-3
    for e in sorted({0, 1, E // 2, E - 1}):
        ref = pb.condense(e)["S"]
        assert np.linalg.norm(got[e] - ref) <= tol * np.linalg.norm(ref), e
    # switched off: a later linearization leaves the buffer alone
    H.hdg_set_element_block_output(run.h, None)
    SK.zero_()
    run.linearize()
    torch.cuda.synchronize()
    assert SK.abs().max().item() == 0.0
    run.close()


def test_tet_element_blocks_match_oracle(H):
    from tests.test_gpu_tet import mesh_case, setup
    prob, pb, h, dev = setup(H, mesh_case(1))
    try:
        L = H.hdg_tet_layout(h)
        ts = np.diff(L["hoff"])[L["e2f"]].sum(1)
        off = np.concatenate([[0], np.cumsum(ts.astype(np.int64) ** 2)])
        SK = torch.zeros(int(off[-1]), dtype=torch.float64, device="cuda")
        H.hdg_set_element_block_output(h, SK)
        H.hdg_linearize_condense(h, dev["U"], dev["Q"], dev["UH"], dev["Ustar"], None, prob.dt, prob.a_ii)
        assert H.hdg_status(h) == H.HDG_OK
        got = SK.cpu().numpy()
        for e in range(len(ts)):
            ref = pb.condense(e)["S"]
            blk = got[off[e]:off[e + 1]].reshape(ts[e], ts[e])
            assert np.linalg.norm(blk - ref) <= 1e-11 * np.linalg.norm(ref), e
    finally:
        H.hdg_destroy(h)


def test_tet_mixed_element_blocks_match_oracle(H):
    """The tetrahedral mixed form (tensor-core contraction and Schur product, FP32
    triangular solves, FP64 interior LU) against the oracle's FP64 condensation of
    every other element: 1e-4 relative per element in the Frobenius norm."""
    from tests.test_gpu_tet import mesh_case, setup
    prob, pb, h, dev = setup(H, mesh_case(1))
    try:
        H.hdg_set_params(h, tau=prob.tau, precision=H.HDG_PREC_MIXED)
        L = H.hdg_tet_layout(h)
        ts = np.diff(L["hoff"])[L["e2f"]].sum(1)
        off = np.concatenate([[0], np.cumsum(ts.astype(np.int64) ** 2)])
        SK = torch.zeros(int(off[-1]), dtype=torch.float32, device="cuda")
        H.hdg_set_element_block_output(h, SK)
        H.hdg_linearize_condense(h, dev["U"], dev["Q"], dev["UH"], dev["Ustar"], None, prob.dt, prob.a_ii)
        assert H.hdg_status(h) == H.HDG_OK
        got = SK.double().cpu().numpy()
        errs = []
        for e in range(0, len(ts), 2):                # every other element: all degrees, curved and affine
            ref = pb.condense(e)["S"]
            blk = got[off[e]:off[e + 1]].reshape(ts[e], ts[e])
            errs.append(np.linalg.norm(blk - ref) / np.linalg.norm(ref))
        assert max(errs) < 1e-4, max(errs)
        assert max(errs) > 0.0                      # FP32 arithmetic is visible: not an FP64 copy
    finally:
        H.hdg_destroy(h)
