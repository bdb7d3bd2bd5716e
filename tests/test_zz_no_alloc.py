"""The allocation-free linearize entry point against the allocating one (GPU).

hdg_linearize_condense_static serves callers that may not allocate device
memory after set-up; its scratch is a fixed device array inside the library.
This file is collected last so that a stop-at-first-failure run has already
run every other test; it also passes alone in a fresh process.
"""
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


@pytest.mark.parametrize("make", [lambda: synth.config2(n=4), lambda: synth.config3(n=3)],
                         ids=["hex-p2-64-elements", "hex-p3-27-elements"])
def test_static_scratch_matches_allocating_entry_point(make):
    from paper_2608_27863_gb300 import hdg as H
    P = make()
    run = GpuRun(P).linearize()                      # allocating entry point
    ref_vals, ref_g = run.blocks(), run.rhs()
    assert H.hdg_status(run.h) == 0
    for _ in range(2):                               # two calls in a row through the C-ABI
        rc = H.lib().hdg_linearize_condense_static(
            run.h, H._ptr(run.U), H._ptr(run.Q), H._ptr(run.UH), H._ptr(run.Ustar), H._ptr(run.nu),
            float(P.dt), float(P.a_ii))
        assert rc == H.HDG_OK, H.hdg_last_error(run.h)
        assert H.hdg_status(run.h) == 0
        vals, g = run.blocks(), run.rhs()
        for b in range(vals.shape[0]):
            assert np.linalg.norm(vals[b] - ref_vals[b]) <= TOL * np.linalg.norm(ref_vals[b]), b
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
