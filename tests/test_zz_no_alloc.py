"""The allocation-free linearize entry point against the allocating one (GPU).

hdg_linearize_condense_static serves callers that may not allocate device
memory after set-up; its scratch is a fixed device array inside the library.
This file is collected last so that a stop-at-first-failure run has already
run every other test; it also passes alone in a fresh process.
"""
import os

import numpy as np
import pytest

import synth
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


def _tau1():
    P = synth.config2(n=4)
    P.tau_mode = 1
    return P


def _plate():
    P = synth.config5(4, 6, 3, 2)
    P.nu = synth.synthetic_nu(P.mesh, P.p, 17, 2e-3)    # a positive AV field: the nu terms are exercised
    return P


def _static(H, run, P):
    return H.lib().hdg_linearize_condense_static(
        run.h, H._ptr(run.U), H._ptr(run.Q), H._ptr(run.UH), H._ptr(run.Ustar), H._ptr(run.nu),
        float(P.dt), float(P.a_ii))


# scratch: the handle's scratch budget at creation (None: the default); the static
# path's chunk (45 hex p=2 elements) is then larger than the handle's own chunk
CASES = [
    (lambda: synth.config2(n=4), None),
    (lambda: synth.config3(n=3), None),
    (_tau1, 5 * 1024 * 1024),
    (_plate, 5 * 1024 * 1024),
]


@pytest.mark.parametrize("make,scratch", CASES,
                         ids=["hex-p2-64-elements", "hex-p3-27-elements", "hex-p2-tau-uhat-small-handle-chunk",
                              "plate-p2-walls-inflow-outflow-av-small-handle-chunk"])
def test_static_scratch_matches_allocating_entry_point(make, scratch):
    from paper_2608_27863_gb300 import hdg as H
    P = make()
    if scratch is not None:
        os.environ["HDG_SCRATCH_BYTES"] = str(scratch)
    try:
        run = GpuRun(P).linearize()                  # allocating entry point
    finally:
        os.environ.pop("HDG_SCRATCH_BYTES", None)
    ref_vals, ref_g = run.blocks(), run.rhs()
    assert H.hdg_status(run.h) == 0
    for _ in range(2):                               # two calls in a row through the C-ABI
        rc = _static(H, run, P)
        assert rc == H.HDG_OK, H.hdg_last_error(run.h)
        assert H.hdg_status(run.h) == 0
        vals, g = run.blocks(), run.rhs()
        scale = np.mean([np.linalg.norm(r) for r in ref_vals])
        for b in range(vals.shape[0]):
            nr = np.linalg.norm(ref_vals[b])
            assert np.linalg.norm(vals[b] - ref_vals[b]) <= TOL * (nr if nr > 0 else scale), b
        assert np.linalg.norm(g - ref_g) <= TOL * np.linalg.norm(ref_g)
    run.close()


def test_static_entry_point_needs_reserved_storage():
    from paper_2608_27863_gb300 import hdg as H
    P = synth.config2(n=3)
    run = GpuRun(P)
    args = (run.h, H._ptr(run.U), H._ptr(run.Q), H._ptr(run.UH), H._ptr(run.Ustar), H._ptr(run.nu),
            float(P.dt), float(P.a_ii))
    assert H.lib().hdg_linearize_condense_static(*args) == H.HDG_EINVAL
    assert "reserve" in H.hdg_last_error(run.h)
    H.hdg_reserve(run.h, H.HDG_PREC_FP64)
    assert H.lib().hdg_linearize_condense_static(*args) == H.HDG_OK
    vals = run.blocks()
    ref = GpuRun(P).linearize()
    rv = ref.blocks()
    assert max(np.linalg.norm(vals[b] - rv[b]) / np.linalg.norm(rv[b]) for b in range(0, len(rv), 7)) <= TOL
    ref.close()
    run.close()


def test_static_entry_point_refuses_what_the_allocating_one_refuses():
    """Unset boundary data and a mixed-precision handle are refused before any launch."""
    import torch
    from paper_2608_27863_gb300 import hdg as H
    P = _plate()
    m = P.mesh
    h = H.hdg_create(m.dim, m.vert_xyz, m.elem_vert, m.periodic_map, m.bnd_tag, P.p, P.gamma, P.re, P.pr, P.mach)
    try:
        H.hdg_reserve(h, H.HDG_PREC_FP64)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        U, Q, UH, Us, nu = t(P.U), t(P.Q), t(P.UH), t(P.Ustar), t(P.nu)
        call = lambda: H.lib().hdg_linearize_condense_static(h, H._ptr(U), H._ptr(Q), H._ptr(UH), H._ptr(Us),
                                                             H._ptr(nu), float(P.dt), float(P.a_ii))
        assert call() == H.HDG_EINVAL and "tag 1" in H.hdg_last_error(h)
        H.hdg_set_bc_state(h, 1, P.ubc)
        assert call() == H.HDG_EINVAL and "tag 3" in H.hdg_last_error(h)
        H.hdg_set_bc_state(h, 3, np.array([P.twall]))
        H.hdg_set_params(h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s,
                         precision=H.HDG_PREC_MIXED)
        assert call() == H.HDG_EUNSUPPORTED
        H.hdg_set_params(h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s,
                         precision=H.HDG_PREC_FP64)
        assert call() == H.HDG_OK, H.hdg_last_error(h)
        assert H.hdg_status(h) == 0
    finally:
        H.hdg_destroy(h)
