"""Mixed-precision form (FP64 LU, residual and Arnoldi; FP32 blocks) on the GPU.

Its condensed blocks are an inexact linearization: they are compared with the
FP64 path (which matches the oracle to 1e-11) and their error is reported and
bounded by the FP32 rounding level times the blocks' conditioning.  The
Newton iteration, whose residual is always evaluated in FP64, must reach the
same converged state as the FP64 iteration.
"""
import numpy as np
import pytest

import synth
from tests.helpers import GpuRun

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_27863_gb300 import build
    build.build()


def blocks_of(run, mixed):
    import torch
    s = run.sizes
    n = s["nnzb"] * s["block"] ** 2
    from paper_2608_27863_gb300 import hdg as H
    v = torch.empty(n, dtype=torch.float32 if mixed else torch.float64, device="cuda")
    H.hdg_get_blocks(run.h, v)
    torch.cuda.synchronize()
    return v.double().cpu().numpy().reshape(s["nnzb"], s["block"], s["block"]).transpose(0, 2, 1)


@pytest.mark.parametrize("make", [synth.config1, lambda: synth.config2(n=3), lambda: synth.config3(n=3),
                                  lambda: synth.tiny(2, 3, visc_law=1, av=2e-3)],
                         ids=["quad-p2", "hex-p2", "hex-p3-av", "quad-p3-av"])
def test_mixed_blocks_against_fp64(make, record_property):
    from paper_2608_27863_gb300 import hdg as H
    P = make()
    run = GpuRun(P)
    run.linearize()
    ref = blocks_of(run, False)
    gref = run.rhs()
    H.hdg_set_params(run.h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s,
                     precision=H.HDG_PREC_MIXED)
    run.linearize()
    assert H.hdg_status(run.h) == 0
    mix = blocks_of(run, True)
    g = run.rhs()
    errs = [np.linalg.norm(mix[b] - ref[b]) / np.linalg.norm(ref[b]) for b in range(ref.shape[0])]
    gerr = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    record_property("max_block_rel_err", float(max(errs)))
    record_property("rhs_rel_err", float(gerr))
    assert max(errs) < 1e-3, max(errs)
    assert gerr < 1e-3, gerr
    run.close()


@pytest.mark.parametrize("make", [synth.config1, lambda: synth.config2(n=4)], ids=["quad-p2", "hex-p2"])
def test_mixed_newton_reaches_fp64_state(make, record_property):
    import torch
    from paper_2608_27863_gb300 import hdg as H
    P = make()
    a = GpuRun(P)
    na, ga, ha = H.hdg_newton(a.h, a.U, a.Q, a.UH, a.Ustar, a.nu, P.dt, P.a_ii, tol=1e-11, max_newton=10,
                              restart=40, max_gmres=800, gmres_rtol=1e-12)
    b = GpuRun(P)
    H.hdg_set_params(b.h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s,
                     precision=H.HDG_PREC_MIXED)
    nb, gb, hb = H.hdg_newton(b.h, b.U, b.Q, b.UH, b.Ustar, b.nu, P.dt, P.a_ii, tol=1e-11, max_newton=30,
                              restart=40, max_gmres=800, gmres_rtol=1e-12)
    record_property("fp64_history", [float(v) for v in ha])
    record_property("mixed_history", [float(v) for v in hb])
    assert ha[-1] <= 1e-11 and hb[-1] <= 1e-11
    # the same root of the FP64 stage residual, up to the residual tolerance
    for x, y, tol in ((a.U, b.U, 1e-10), (a.UH, b.UH, 1e-10), (a.Q, b.Q, 1e-9)):
        x, y = x.cpu().numpy(), y.cpu().numpy()
        assert np.linalg.norm(x - y) <= tol * np.linalg.norm(x)
    a.close()
    b.close()


@pytest.mark.parametrize("make", [synth.config1, lambda: synth.config2(n=3), lambda: synth.config3(n=3)],
                         ids=["quad-p2", "hex-p2", "hex-p3-av"])
def test_tensor_core_schur_variants(make, record_property):
    """The tcgen05 Schur product (TF32, 3xTF32) against the FP32 SIMT product and FP64."""
    from paper_2608_27863_gb300 import hdg as H
    P = make()
    run = GpuRun(P)
    run.linearize()
    ref = blocks_of(run, False)
    out = {}
    for prec in (H.HDG_PREC_MIXED, H.HDG_PREC_MIXED_TF32, H.HDG_PREC_MIXED_3XTF32):
        H.hdg_set_params(run.h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s, precision=prec)
        run.linearize()
        assert H.hdg_status(run.h) == 0, H.hdg_last_error(run.h)
        out[prec] = blocks_of(run, True)
    rel = lambda x, y: max(np.linalg.norm(x[b] - y[b]) / np.linalg.norm(y[b]) for b in range(y.shape[0]))
    e_simt = rel(out[H.HDG_PREC_MIXED], ref)
    e_tf32 = rel(out[H.HDG_PREC_MIXED_TF32], ref)
    e_3x = rel(out[H.HDG_PREC_MIXED_3XTF32], ref)
    d_3x = rel(out[H.HDG_PREC_MIXED_3XTF32], out[H.HDG_PREC_MIXED])
    record_property("err_simt_fp32", float(e_simt))
    record_property("err_tf32", float(e_tf32))
    record_property("err_3xtf32", float(e_3x))
    assert d_3x < 1e-4, d_3x          # 3xTF32 tracks the FP32 product
    assert e_3x < 1e-3 and e_tf32 < 3e-2
    run.close()


def test_tensor_core_newton_3xtf32():
    from paper_2608_27863_gb300 import hdg as H
    P = synth.config2(n=4)
    a = GpuRun(P)
    H.hdg_newton(a.h, a.U, a.Q, a.UH, a.Ustar, a.nu, P.dt, P.a_ii, tol=1e-11, max_newton=10, restart=40,
                 max_gmres=800, gmres_rtol=1e-12)
    b = GpuRun(P)
    H.hdg_set_params(b.h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s,
                     precision=H.HDG_PREC_MIXED_3XTF32)
    nb, gb, hb = H.hdg_newton(b.h, b.U, b.Q, b.UH, b.Ustar, b.nu, P.dt, P.a_ii, tol=1e-11, max_newton=30,
                              restart=40, max_gmres=800, gmres_rtol=1e-12)
    assert hb[-1] <= 1e-11
    x, y = a.UH.cpu().numpy(), b.UH.cpu().numpy()
    assert np.linalg.norm(x - y) <= 1e-10 * np.linalg.norm(x)
    a.close()
    b.close()


def test_autotune_mixed_picks_fp32_accurate_schur():
    from paper_2608_27863_gb300 import hdg as H
    P = synth.config2(n=3)
    run = GpuRun(P)
    H.hdg_set_params(run.h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s,
                     precision=H.HDG_PREC_MIXED)
    rep = H.hdg_autotune(run.h, run.U, run.Q, run.UH, run.Ustar, run.nu, P.dt, P.a_ii, reps=1)
    assert {c[2] for c, _ in rep["candidates"]} == {0, 2} and rep["schur_mode"] in (0, 2)
    # an explicit TF32 request is not overridden
    H.hdg_set_params(run.h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s,
                     precision=H.HDG_PREC_MIXED_TF32)
    rep = H.hdg_autotune(run.h, run.U, run.Q, run.UH, run.Ustar, run.nu, P.dt, P.a_ii, reps=1)
    assert len(rep["candidates"]) == 12 and rep["schur_mode"] == 1
    assert {c[3] for c, _ in rep["candidates"]} == {0, 1, 2} and {c[6] for c, _ in rep["candidates"]} == {0, 1}
    assert {c[0] for c, _ in rep["candidates"] if c[6] == 1} == {16, 8}
    run.close()


@pytest.mark.parametrize("make", [lambda: synth.config2(n=3), lambda: synth.config3(n=3)], ids=["hex-p2", "hex-p3"])
def test_tensor_core_contraction_matches_simt(make):
    """The 3xTF32 tcgen05 volume contraction, the FP32 sum-factorised one and the
    dense FP32 SIMT one agree to FP32 accuracy."""
    import torch
    from paper_2608_27863_gb300 import hdg as H
    P = make()
    out = {}
    for bm in (0, 1, 2):
        run = GpuRun(P)
        H.hdg_set_params(run.h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s,
                         precision=H.HDG_PREC_MIXED)
        H.hdg_set_tuning(run.h, schur_mode=0, blocks_mode=bm)
        run.linearize()
        assert H.hdg_status(run.h) == 0
        s = run.sizes
        v = torch.empty(s["nnzb"] * s["block"] ** 2, dtype=torch.float32, device="cuda")
        H.hdg_get_blocks(run.h, v)
        out[bm] = (v.cpu().numpy().astype(np.float64), run.rhs())
        run.close()
    v0, g0 = out[0]
    for bm in (1, 2):
        v1, g1 = out[bm]
        assert np.linalg.norm(v1 - v0) <= 2e-6 * np.linalg.norm(v0), bm
        assert np.linalg.norm(g1 - g0) <= 2e-6 * np.linalg.norm(g0), bm



@pytest.mark.parametrize("make", [lambda: synth.config2(n=3), lambda: synth.config3(n=3),
                                  lambda: synth.tiny(2, 3, periodic=(True, False), visc_law=1, av=1e-3)],
                         ids=["hex-p2", "hex-p3", "quad-p3-dirichlet"])
def test_split_elimination_matches_fused(make):
    """FP64 interior LU + FP32 triangular solves give the fused elimination's
    condensed system to FP32 accuracy, and the same recovery."""
    import torch
    from paper_2608_27863_gb300 import hdg as H
    P = make()
    out = {}
    for split, nb in ((0, 16), (1, 16), (1, 8)):
        run = GpuRun(P)
        H.hdg_set_params(run.h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s,
                         precision=H.HDG_PREC_MIXED_3XTF32)
        H.hdg_set_tuning(run.h, elim_nb=nb, schur_mode=2, blocks_mode=1 if P.mesh.dim == 3 else 0,
                         elim_mixed_split=split)
        run.linearize()
        assert H.hdg_status(run.h) == 0
        s = run.sizes
        v = torch.empty(s["nnzb"] * s["block"] ** 2, dtype=torch.float32, device="cuda")
        H.hdg_get_blocks(run.h, v)
        rng = np.random.default_rng(2)
        dq, du = run.recover(rng.normal(size=P.UH.shape) * 1e-3)
        out[(split, nb)] = (v.cpu().numpy().astype(np.float64), run.rhs(), du)
        run.close()
    v0, g0, u0 = out[(0, 16)]
    for key in ((1, 16), (1, 8)):
        v1, g1, u1 = out[key]
        assert np.linalg.norm(v1 - v0) <= 1e-5 * np.linalg.norm(v0)
        assert np.linalg.norm(g1 - g0) <= 1e-5 * np.linalg.norm(g0)
        assert np.linalg.norm(u1 - u0) <= 1e-5 * np.linalg.norm(u0)
