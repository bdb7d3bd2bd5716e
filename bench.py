#!/usr/bin/env python
"""Benchmark: HDG linearize + condense throughput on GB300.

One step is one pass of the whole hot path over the workload: per-element
quadrature-point fluxes and Jacobians, contraction into the element blocks,
bordered elimination (interior LU, solves, Schur complement), assembly of the
block-sparse trace system, one trace matvec and the interior recovery.

Default workload: the batched tetrahedral mesh, 30 x 20 x 28 Kuhn cells =
100,800 tetrahedra with a seeded mix of degrees 1..4, a quadratic (curved)
wall layer with wall-normal stretching 1.2 and aspect ratios up to 1e3,
perturbed freestream at M = 0.5, Re = 1e5; FP64, one persistent launch for
the whole mix.  The same process times the mixed form on the same mesh and
compares Newton to ||F|| <= 1e-8 in both forms.  Inputs are resident in HBM
for ``value``; ``e2e`` repeats the step through the C-ABI from pinned host
buffers.  ``--workload`` selects the hexahedral workloads (16^3 hex p = 2,
24^3 hex p = 3 with AV, the flat plate, ...).

``--impl reference`` times the FP64 CPU oracle on the host cores instead (the
only other place this file runs ``oracle/``), on a bounded element sample.
Under torchrun each rank runs an independent replica (elements are
independent; no data-path collective) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HDG linearize+condense elements/s & % of FP64/TC peak; mixed vs FP64 at tol"

# DRAM bytes (read + write) per element of the dominant kernel, from one ncu
# capture of the unchanged kernel on the 8^3 hex p=2 case (512 elements, above
# L2); every CTA works on its own element, so traffic scales with the element
# count of a launch.
# Keyed by (kernel, d, p, elimination panel width).
DRAM_BYTES_PER_ELEMENT = {("elim", 3, 2, 16): 16.45e6, ("elim", 3, 2, 8): 30.84e6,
                          # FP64 element blocks, sum-factorised: k_blocks_sf (0.377 GB) + the face-term
                          # pass k_blocks (0.936 GB) on the 512-element 8^3 launch
                          ("blocks_sf", 3, 2, 0): (0.3775e9 + 0.9359e9) / 512}
# The persistent tetrahedral kernel k_tet_linearize<double>: 87.5 GB (read + write) in one
# ncu-captured launch over the 3,600 elements of the 10 x 20 x 3 mesh, whose degree mix and
# curved fraction come from the same seeded generator as the 100,800-element mesh; the
# traffic is the per-CTA workspace streamed per element, so it scales with the elements.
TET_DRAM_BYTES_PER_ELEMENT = 87.5e9 / 3600
L2_BYTES = 129 * 1024 * 1024

# fn/kw: the synth generator; mixed_only: the FP64 arrays would not fit in HBM, so only
# the mixed form is timed; av: (c_av, h_m) of an artificial-viscosity field computed
# from the state on the device before timing; cpu: a smaller mesh of the same elements
# and physics from which the oracle's element sample is drawn.
WORKLOADS = {
    "hex-p2-16^3-tgv": dict(fn="config2", kw={}),
    "hex-p2-8^3-tgv": dict(fn="config2", kw={"n": 8}),
    "hex-p3-24^3-tgv-av": dict(fn="config3", kw={}),
    "quad-p2-8x8": dict(fn="config1", kw={}),
    "hex-p3-64x48x32-plate": dict(fn="config5", kw={}, mixed_only=True, av=(2e-3, 0.1 / 48),
                                  cpu=dict(fn="config5", kw={"nx": 6, "ny": 8, "nz": 4})),
    "hex-p2-8x12x6-plate": dict(fn="config5", kw={"nx": 8, "ny": 12, "nz": 6, "p": 2}, av=(2e-3, 0.1 / 12)),
    # curved anisotropic tetrahedra, degrees 1..4 per element (seeded), 6 Kuhn tets per cell
    "tet-p1to4-30x20x28-curved": dict(kind="tet", kw={}),
    "tet-p1to4-10x20x6-curved": dict(kind="tet", kw={"nx": 10, "nz": 6}),
    "tet-p1to4-10x20x3-curved": dict(kind="tet", kw={"nx": 10, "nz": 3}),
}
DEFAULT_WORKLOAD = "tet-p1to4-30x20x28-curved"


def make_tet_problem(name, host_layout=None):
    """Mesh, physics and packed seeded state of a tetrahedral workload.  The trace
    sizes come from the library's layout when given (GPU leg), else from the
    oracle's connectivity (CPU leg); both give the same numbers."""
    import numpy as np
    from synth import tetmesh as tm
    m = tm.config4_mesh(**WORKLOADS[name]["kw"])
    P = tm.config4_problem(m)
    if host_layout is None:
        from oracle.tet import TetConnectivity
        nfp = TetConnectivity(m).nfp
    else:
        nfp = np.diff(host_layout["hoff"]) // 5
    fun = tm.sinusoids(P.gamma, P.mach, 3, 1e-3)
    P.U, P.Q, P.UH, P.Ustar = tm.packed_state(m, fun, nfp, P.ubc, 7)
    return P, m


def cpu_model():
    """The host CPU as the OS reports it (model name, or the Arm part and implementer)."""
    try:
        info = open("/proc/cpuinfo").read()
    except OSError:
        return None
    for key in ("model name", "Model name"):
        for line in info.splitlines():
            if line.startswith(key):
                return line.split(":", 1)[1].strip()
    fields = {}
    for line in info.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            fields.setdefault(k.strip(), v.strip())
    if "CPU part" in fields:
        parts = {"0xd4f": "Neoverse-V2", "0xd40": "Neoverse-V1", "0xd0c": "Neoverse-N1"}
        return "Arm %s (implementer %s, part %s)" % (parts.get(fields["CPU part"], "core"),
                                                     fields.get("CPU implementer", "?"), fields["CPU part"])
    return None


def hbm_peak_gbs():
    """Measured copy bandwidth of the GB300s (GB/s) and its source."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json (measured)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


def tet_recover_bytes(layout, elem_p):
    """Bytes the interior recovery must move per launch: per element the interior
    rows' trace part and right-hand side NU (t + 1), the upper triangle of the
    interior factor NU (NU + 1) / 2, the recovery data G, H, dq0 (3 Np^2 +
    3 Np sum nfp + 3 NU), the element's trace values t; writes dU, dQ (4 NU)."""
    import numpy as np
    fp = layout["face_p"][layout["e2f"]]
    Np = (elem_p + 1) * (elem_p + 2) * (elem_p + 3) // 6
    sfp = ((fp + 1) * (fp + 2) // 2).sum(1)
    NU, t = 5 * Np, 5 * sfp
    words = NU * (t + 1) + NU * (NU + 1) / 2 + 3 * Np * Np + 3 * Np * sfp + 3 * NU + t + 4 * NU
    return float(8 * words.sum())


def hex_recover_bytes(d, p, E):
    """The same for quad / hex elements: interior rows NU (NT + 1) + NU (NU + 1) / 2,
    dq0 (NQV), the element trace NT; writes dU, dQ (NU + NQV)."""
    m, Np = d + 2, (p + 1) ** d
    NU, NQV, NT = m * Np, d * m * Np, 2 * d * m * (p + 1) ** (d - 1)
    return 8.0 * E * (NU * (NT + 1) + NU * (NU + 1) / 2 + NQV + NT + NU + NQV)


def tet_flops(layout, elem_p):
    """Algorithmic FP64 flops per element of the tetrahedral linearize + condense kernel:
    point values and lifting operators, contraction (element and trace rows, with the
    per-point column variations), and the bordered elimination."""
    import numpy as np
    E = len(elem_p)
    fp = layout["face_p"][layout["e2f"]]                      # [E][4]
    Np = (elem_p + 1) * (elem_p + 2) * (elem_p + 3) // 6
    Nq = (elem_p + 2) ** 3
    nfp = (fp + 1) * (fp + 2) // 2
    nfq = (fp + 2) ** 2
    sfp, sfq = nfp.sum(1), nfq.sum(1)
    Nc = Np + sfp
    NU, t = 5 * Np, 5 * sfp
    lift = 3 * Np * Np * Nq + 9 * Np * Np * Nq + 9 * Np * sfp * nfq.max(1) + Np ** 3 / 3 + 6 * Nc * Np * Np \
        + 2 * 15 * Np * (Np + sfp) + 2 * 3 * (Nq + sfq) * Nc * Np
    contr = 2 * 25 * Np * Nc * (3 * Nq + sfq) + 2 * 25 * (nfp * nfq).sum(1) * Nc \
        + 25 * Nc * (3 * Nq * 8 + sfq * 10 + sfq * 10)
    elim = np.zeros(E)
    for e in range(E):
        k = np.arange(NU[e])
        NR = NU[e] + t[e]
        elim[e] = np.sum(2.0 * (NR - k - 1) * (NR - k) + (NR - k - 1))
    return {"lift": lift, "contraction": contr, "elim": elim, "total": lift + contr + elim}


def run_tet(args, rank, world, local_rank):
    """Tetrahedral workload (mixed degree, curved and affine elements, one persistent
    FP64 launch): linearize + condense, trace matvec and recovery per step."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2608_27863_gb300 import build as B
    from paper_2608_27863_gb300 import hdg as H

    pool = None
    ncores = os.cpu_count() or 1
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = oracle_pool(args.workload, ncores)      # before the first GPU call
    torch.cuda.set_device(local_rank)
    B.build()
    peaks, _ = H.hdg_measure_peaks()           # hand-written pipe probes on this GPU (untimed)
    from synth import tetmesh as tm
    m0 = tm.config4_mesh(**WORKLOADS[args.workload]["kw"])
    hh = H.hdg_create_tet(m0.vert_xyz, m0.elem_vert, m0.periodic_map, m0.bnd_tag, m0.elem_p, m0.geo, 1.4, 1e5,
                          0.72, 0.5, host_only=True)
    layout = H.hdg_tet_layout(hh)
    H.hdg_destroy(hh)
    P, m = make_tet_problem(args.workload, host_layout=layout)
    h = H.hdg_create_tet(m.vert_xyz, m.elem_vert, m.periodic_map, m.bnd_tag, m.elem_p, m.geo, P.gamma, P.re, P.pr,
                         P.mach)
    H.hdg_set_params(h, tau=P.tau)
    H.hdg_set_bc_state(h, 1, P.ubc)
    sizes = H.hdg_tet_query(h)
    stream = torch.cuda.current_stream()
    H.hdg_set_stream(h, stream.cuda_stream)
    dev = torch.device("cuda", local_rank)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    U, Q, UH, Us = t(P.U), t(P.Q), t(P.UH), t(P.Ustar)
    x = t(np.random.default_rng(rank).normal(size=P.UH.shape))
    y = torch.empty_like(UH)
    dQ, dU = torch.empty_like(Q), torch.empty_like(U)
    flush = torch.empty(2 * L2_BYTES // 8, dtype=torch.float64, device=dev)

    def step():
        H.hdg_linearize_condense(h, U, Q, UH, Us, None, P.dt, P.a_ii)
        H.hdg_trace_matvec(h, x, y)
        H.hdg_recover_interior(h, y, dQ, dU)

    def timed(nsteps, nwarm):
        for _ in range(nwarm):
            step()
        torch.cuda.synchronize()
        if H.hdg_status(h) != 0:
            raise RuntimeError("device status: " + H.hdg_last_error(h))
        H.hdg_profile_read(h)
        H.hdg_profile(h, True)
        if world > 1:
            dist.barrier()
        times = []
        with ClockSampler(local_rank) as clk:
            for _ in range(nsteps):
                flush.fill_(1.0)
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record(stream)
                step()
                e.record(stream)
                e.synchronize()
                times.append(s.elapsed_time(e))
        torch.cuda.synchronize()
        prof = H.hdg_profile_read(h)
        H.hdg_profile(h, False)
        return max_over_ranks(sum(times), world, dev), prof, clk.summary()

    def tune():
        # the project's autotuner picks the elimination panel width of the persistent kernel (untimed)
        if args.no_autotune or args.tuning:
            nb = 16
            for item in (args.tuning or "").split(","):
                if item.startswith("elim_nb="):
                    nb = int(item.split("=")[1])
            H.hdg_set_tuning(h, elim_nb=nb)
            return {"elim_nb": nb, "fixed": True}
        rep = H.hdg_autotune(h, U, Q, UH, Us, None, P.dt, P.a_ii, reps=1)
        return {"elim_nb": rep["elim_nb"], "candidates_ms": [c[1] for c in rep["candidates"]]}

    tuning = {}
    H.hdg_set_params(h, tau=P.tau, precision=H.HDG_PREC_FP64)
    tuning["fp64"] = tune()
    t_ms, prof, clocks = timed(args.steps, args.warmup)
    # the mixed leg and the end-to-end leg are bounded (at most 5 and 3 steps) so that a
    # long headline run stays within minutes; their step counts are reported
    n_mixed, n_e2e = min(args.steps, 5), min(args.steps, 3)
    if not args.no_mixed:
        H.hdg_set_params(h, tau=P.tau, precision=H.HDG_PREC_MIXED)
        tuning["mixed"] = tune()
        tm_ms, prof_m, clocks_m = timed(n_mixed, min(args.warmup, 2))
        H.hdg_set_params(h, tau=P.tau, precision=H.HDG_PREC_FP64)
        H.hdg_set_tuning(h, elim_nb=tuning["fp64"]["elim_nb"])
    # end to end from pinned host memory
    hU, hQ, hUH, hUs = (torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (P.U, P.Q, P.UH, P.Ustar))
    hdQ = torch.empty(dQ.shape, dtype=torch.float64).pin_memory()
    hdU = torch.empty(dU.shape, dtype=torch.float64).pin_memory()
    h2d = sum(a.numel() * 8 for a in (hU, hQ, hUH, hUs))
    d2h = (hdQ.numel() + hdU.numel()) * 8
    e2e_ms = 0.0
    for _ in range(n_e2e):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        U.copy_(hU, non_blocking=True)
        Q.copy_(hQ, non_blocking=True)
        UH.copy_(hUH, non_blocking=True)
        Us.copy_(hUs, non_blocking=True)
        step()
        hdQ.copy_(dQ, non_blocking=True)
        hdU.copy_(dU, non_blocking=True)
        e.record(stream)
        e.synchronize()
        e2e_ms += s.elapsed_time(e)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    cpu = None
    check_ids, check_refs = None, None
    if pool is not None:
        rate, n_done, secs = oracle_rate(pool, ncores, m.n_elem, args.cpu_seconds, 100)
        check_ids = oracle_check_elements(elem_p=m.elem_p)
        check_refs = pool.map(_worker_schur, check_ids)
        pool.close()
        cpu = {"value": rate, "unit": "elements/s", "cores": ncores, "cpu_model": cpu_model(), "kind": "oracle",
               "sample": "%d seeded elements of the workload in %.1f s: per-element residual, complex-step "
                         "Jacobian, dense FP64 LU of the (q,u) block and Schur complement" % (n_done, secs)}
    oracle_check = None
    if check_ids is not None:
        # per-element S^K of both forms against the oracle's condensation of the same elements (untimed)
        ts = np.diff(layout["hoff"])[layout["e2f"]].sum(1).astype(np.int64)
        offs = np.concatenate([[0], np.cumsum(ts ** 2)])

        def tet_prec(prec):
            H.hdg_set_params(h, tau=P.tau, precision=prec)
            H.hdg_set_tuning(h, elim_nb=tuning["mixed" if prec != H.HDG_PREC_FP64 else "fp64"]["elim_nb"])

        run1 = lambda: H.hdg_linearize_condense(h, U, Q, UH, Us, None, P.dt, P.a_ii)
        precs = {"fp64": (H.HDG_PREC_FP64, tet_prec, run1)}
        if not args.no_mixed:
            precs["mixed"] = (H.HDG_PREC_MIXED, tet_prec, run1)
        oracle_check = element_block_errors(H, h, torch, check_ids, offs, ts, check_refs, precs)
        oracle_check = {"what": "relative Frobenius error of the per-element Schur complement S^K against the "
                                "FP64 CPU oracle's condensation of the same element",
                        "elements": check_ids, "degrees": [int(m.elem_p[e]) for e in check_ids], **oracle_check}
        H.hdg_set_params(h, tau=P.tau, precision=H.HDG_PREC_FP64)
        H.hdg_set_tuning(h, elim_nb=tuning["fp64"]["elim_nb"])
    E = m.n_elem
    fl = tet_flops(layout, m.elem_p.astype(np.int64))
    kern = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
            for k, v in prof.items() if v[1]}
    lin_ms = prof["elim"][0] / max(prof["elim"][1], 1)
    achieved = fl["total"].sum() / (lin_ms * 1e-3) / 1e12
    smmax = clocks.get("sm_max_mhz") or 2070.0
    peak = fp64_peak_derived(smmax)
    counts = np.bincount(m.elem_p, minlength=5)[1:]
    mixed = None if args.no_mixed else {"value": replica_throughput(world, E, n_mixed, tm_ms), "unit": "elements/s",
             "steps": n_mixed, "ms_per_step": tm_ms / n_mixed,
             "speedup_vs_fp64_step": (t_ms / args.steps) / (tm_ms / n_mixed),
             "kernels": {k: {"ms_per_step": v[0] / n_mixed, "launches_per_step": v[1] / n_mixed}
                         for k, v in prof_m.items() if v[1]},
             "dtype": "fp64 pointwise terms, lifting operators, elimination and residual; fp32 Jacobian "
                      "coefficients, column variations and contraction",
             "clocks": clocks_m}
    if mixed is not None and oracle_check is not None:
        mixed["block_err_vs_oracle"] = oracle_check["mixed"]["max_rel_err"]
    if not args.no_newton and mixed is not None:
        newton = {}
        H.hdg_set_preconditioner(h, H.HDG_PC_SCHWARZ if args.precond == "schwarz" else H.HDG_PC_BLOCKJACOBI)
        for name, prec in (("fp64", H.HDG_PREC_FP64), ("mixed", H.HDG_PREC_MIXED)):
            H.hdg_set_params(h, tau=P.tau, precision=prec)
            H.hdg_set_tuning(h, elim_nb=tuning[name]["elim_nb"])
            U2, Q2, UH2 = U.clone(), Q.clone(), UH.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            nit, git, hist = H.hdg_newton(h, U2, Q2, UH2, Us, None, P.dt, P.a_ii, tol=1e-8, max_newton=10,
                                          restart=100, max_gmres=100, gmres_rtol=1e-6, raise_on_noconv=False)
            torch.cuda.synchronize()
            newton[name] = {"seconds": time.perf_counter() - t0, "newton_iters": nit, "gmres_iters": git,
                            "residual_history": [float(v) for v in hist]}
            newton[name + "_U"] = U2
        newton["state_rel_diff_U"] = float(torch.linalg.norm(newton["mixed_U"] - newton["fp64_U"]) /
                                           torch.linalg.norm(newton["fp64_U"]))
        del newton["mixed_U"], newton["fp64_U"]
        newton["tol"] = 1e-8
        newton["gmres"] = ("restart 100, at most 100 iterations per Newton step, relative tolerance 1e-6, %s" %
                           {"schwarz": "additive Schwarz on element face patches (factors in the system's precision)",
                            "bj": "block-Jacobi"}[args.precond])
        newton["speedup"] = newton["fp64"]["seconds"] / newton["mixed"]["seconds"]
        mixed["newton"] = newton
        H.hdg_set_params(h, tau=P.tau, precision=H.HDG_PREC_FP64)
    if args.dirk and mixed is not None:
        # one SDIRK3 step, 3 stages x n Newton iterations (GMRES(m) each) captured as one CUDA graph,
        # mixed form; the first call captures (after one eager linearization), the second replays
        H.hdg_set_params(h, tau=P.tau, precision=H.HDG_PREC_MIXED)
        H.hdg_set_tuning(h, elim_nb=tuning["mixed"]["elim_nb"])
        A3, b3 = H.sdirk3_tableau()
        U2, Q2, UH2 = U.clone(), Q.clone(), UH.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H.hdg_dirk_step(h, U2, Q2, UH2, None, P.dt, A3, b3, n_newton=args.dirk_newton, m=args.dirk_m,
                        use_graph=True)
        t_first = time.perf_counter() - t0
        t0 = time.perf_counter()
        hist = H.hdg_dirk_step(h, U2, Q2, UH2, None, P.dt, A3, b3, n_newton=args.dirk_newton, m=args.dirk_m,
                               use_graph=True)
        t_replay = time.perf_counter() - t0
        mixed["dirk_step"] = {"stages": 3, "newton_per_stage": args.dirk_newton, "gmres_m": args.dirk_m, "graph": True,
                              "seconds_capture_and_run": t_first, "seconds_replay": t_replay,
                              "residual_history": [[float(v) for v in row] for row in hist]}
        H.hdg_set_params(h, tau=P.tau, precision=H.HDG_PREC_FP64)
    out = {
        "metric": METRIC, "value": replica_throughput(world, E, args.steps, t_ms), "unit": "elements/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "elements_per_gpu": E, "element": "tetrahedron",
                   "degrees": {"p%d" % (i + 1): int(c) for i, c in enumerate(counts)},
                   "curved_elements": sizes["n_curved"], "faces": sizes["n_faces"], "blocks": sizes["nnzb"],
                   "block_values": sizes["n_vals"], "device_bytes": sizes["device_bytes"],
                   "launch": "one persistent launch over a cost-ordered element list",
                   "parallelism": "replicas" if world > 1 else "single", "precision": "fp64",
                   "l2": "flushed between timed steps (256 MiB write)"},
        "roofline": {"bound": "alu", "kernel": "k_tet_linearize", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": TET_DRAM_BYTES_PER_ELEMENT * E / max(prof["elim"][1] / args.steps, 1),
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_tet_linearize "
                                       "launch on the 3,600-element mesh of the same generator, per element, times "
                                       "the elements of one launch",
                     "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x %.0f MHz (derived)" % smmax,
                     "peak_measured": peaks["fp64_fma"], "frac_of_measured": achieved / peaks["fp64_fma"],
                     "peak_measured_source": "DFMA-chain probe (hdg_measure_peaks) in this run",
                     "flops_per_element": float(fl["total"].mean()),
                     "flops_split": {k: float(v.sum()) for k, v in fl.items()}},
        "kernels": kern,
        "recover_roofline": recover_roofline("k_tet_recover", tet_recover_bytes(layout, m.elem_p.astype(np.int64)),
                                             prof["recover"]),
        "mixed": mixed,
        "e2e": {"value": replica_throughput(world, E, n_e2e, e2e_ms), "unit": "elements/s", "steps": n_e2e,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": sum(v[1] for v in prof.values()) / args.steps,
        "clocks": clocks,
        "tuning": tuning,
        "peaks_measured_tflops": peaks,
    }
    if oracle_check is not None:
        out["oracle_check"] = oracle_check
    if cpu is not None:
        out["cpu_baseline"] = cpu
    H.hdg_destroy(h)
    return out


def recover_roofline(kernel, nbytes, prof_entry):
    """HBM roofline of the interior recovery: algorithmic bytes per launch over the
    launch's mean event time."""
    ms, n = prof_entry
    if not n:
        return None
    peak, src = hbm_peak_gbs()
    gbs = nbytes / (ms / n * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "bytes_per_launch": nbytes, "ms_per_launch": ms / n,
            "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak, "peak_source": src}


def make_problem(name, cpu_sample=False):
    import synth
    w = WORKLOADS[name]
    src = w.get("cpu", w) if cpu_sample else w
    return getattr(synth, src["fn"])(**src["kw"])


# ----------------------------------------------------------------------------
# algorithmic FLOP counts per element (the executed reduced-structure counts)
# ----------------------------------------------------------------------------
def ozaki_digits(K):
    """Digit width and count of the tensor-core Schur product for inner size K."""
    b = 8 if 5 * K * 255 ** 2 < 2 ** 24 else 7 if 5 * K * 127 ** 2 < 2 ** 24 else 6
    return b, -(-54 // b)


def flop_counts(d, p, sum_factorised=False, tc_schur=False):
    m, n1, q1 = d + 2, p + 1, p + 2
    Np, Nq, nf, Nfp, Nfq = n1 ** d, q1 ** d, 2 * d, n1 ** (d - 1), q1 ** (d - 1)
    NU, NT = m * Np, nf * m * Nfp
    NR, NC = NU + NT, NU + NT + 1
    elim = sum(2 * (NR - k - 1) * (NC - k - 1) + (NR - k - 1) for k in range(NU))
    schur = 2 * NT * NT * NU                  # the trace-trace part of the trailing updates
    b, s = ozaki_digits(NU)
    pairs = s * (s + 1) // 2                  # digit pairs kept (i + j <= s + 1)
    mt, nt = -(-NT // 128) * 128, -(-NT // 32) * 32
    schur_bf16 = pairs * 2 * mt * nt * (-(-NU // 16) * 16)   # executed BF16 MMA work, padded tiles
    if tc_schur:
        elim -= schur
    NCB = Np + nf * Nfp
    K = d * Nq
    if sum_factorised:       # one 1-D contraction per axis, per column and direction
        axes = q1 * q1 * n1 * q1 + q1 * n1 * n1 * q1 + n1 ** 3 * q1 if d == 3 else q1 * n1 * q1 + n1 * n1 * q1
        contraction = 2 * axes * NCB * d
    else:
        contraction = 2 * Np * NCB * K
    blocks = m * m * (contraction                       # contraction
                      + K * (2 * (1 + d) * Np + nf * Nfp)  # generated operand
                      + nf * (2 * Nfq * NCB * (d + 1) + 2 * Nfp * NCB * Nfq))  # face terms
    out = {"elim": elim, "blocks": blocks, "total": elim + blocks + (schur if tc_schur else 0)}
    if tc_schur:
        out.update(schur=schur, schur_bf16=schur_bf16)
    return out


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU oracle leg (spawned workers, one single-threaded process per core)
# ----------------------------------------------------------------------------
_W = {}


def _worker_init(name):
    sys.path.insert(0, ROOT)
    import numpy as np
    if WORKLOADS[name].get("kind") == "tet":
        from oracle.tet import TetProblem
        _W["pb"] = TetProblem(make_tet_problem(name, host_layout=None)[0])
        return
    from oracle.hdg import Problem
    P = make_problem(name, cpu_sample=True)
    if P.nu is None and "av" in WORKLOADS[name]:
        P.nu = 0.5 * WORKLOADS[name]["av"][0] * np.ones(P.U[:, 0, :].shape)   # AV on: a positive field
    _W["pb"] = Problem(P)


def _worker_condense(e):
    _W["pb"].condense(int(e))
    return 1


def _worker_schur(e):
    """The oracle's condensed element matrix S^K of element e (FP64)."""
    return _W["pb"].condense(int(e))["S"]


def oracle_pool(name, cores):
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(cores, initializer=_worker_init, initargs=(name,))
    for k, v in saved.items():
        if v is None:
            del os.environ[k]
        else:
            os.environ[k] = v
    pool.map(_worker_condense, [0] * cores)  # warm every worker
    return pool


def oracle_check_elements(elem_p=None, n_elem=0):
    """Elements whose S^K the oracle leg also returns: for a mixed-degree mesh the
    first and last element of every degree, else four spread over the mesh."""
    if elem_p is not None:
        import numpy as np
        ids = []
        for p in range(1, int(elem_p.max()) + 1):
            w = np.flatnonzero(elem_p == p)
            if len(w):
                ids += [int(w[0]), int(w[-1])]
        return sorted(set(ids))
    return sorted({0, n_elem // 3, (2 * n_elem) // 3, n_elem - 1})


def element_block_errors(H, h, torch, ids, offs, sizes, refs, precisions):
    """Relative Frobenius error of the library's per-element S^K against the oracle's,
    per precision (one linearization each through hdg_set_element_block_output)."""
    total = int(offs[-1])
    buf = torch.empty(total, dtype=torch.float64, device="cuda")
    out = {}
    for name, (prec, set_prec, run) in precisions.items():
        set_prec(prec)
        sk = buf if prec == H.HDG_PREC_FP64 else buf.view(torch.float32)[:total]
        H.hdg_set_element_block_output(h, sk)
        run()
        torch.cuda.synchronize()
        H.hdg_set_element_block_output(h, None)
        errs = []
        for e, ref in zip(ids, refs):
            t = int(sizes[e])
            got = sk[int(offs[e]):int(offs[e]) + t * t].double().cpu().numpy().reshape(t, t)
            errs.append(float(((got - ref) ** 2).sum() ** 0.5 / max((ref ** 2).sum() ** 0.5, 1e-300)))
        out[name] = {"max_rel_err": max(errs), "per_element": errs}
    del buf
    torch.cuda.empty_cache()
    return out


def oracle_rate(pool, cores, n_elem, seconds, seed):
    """Elements/s of the oracle's per-element linearize + condense on a seeded sample."""
    import synth
    done, t0 = 0, time.perf_counter()
    batch = 0
    while True:   # at least one batch of one element per core
        ids = [int(x) for x in synth.splitmix64(seed + batch, cores) % n_elem]
        done += sum(pool.map(_worker_condense, ids))
        batch += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return done / dt, done, dt


# ----------------------------------------------------------------------------
# GPU leg
# ----------------------------------------------------------------------------
SMS = 152
FP64_FMA_PER_CLK_PER_SM = 2      # measured with a DFMA-chain probe: 1.19 TFLOP/s saturates at 2 per clock


def fp64_peak_derived(sm_max_mhz):
    """FP64 pipe peak from unit counts and the maximum SM clock (TFLOP/s)."""
    return SMS * FP64_FMA_PER_CLK_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12


def fp64_peak_tflops(torch):
    """cuBLAS DGEMM throughput measured in this run (context for the FP64 roofline)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    c = a @ b
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(3):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        c = a @ b
        e.record()
        torch.cuda.synchronize()
        best = min(best, s.elapsed_time(e))
    del a, b, c
    return 2 * n ** 3 / best / 1e9


# ----------------------------------------------------------------------------
# replicas under torchrun: every rank runs the whole workload (elements are
# independent, no data-path collective); the step time is the maximum over ranks
# ----------------------------------------------------------------------------
def max_over_ranks(t_ms, world, device):
    """The largest of the ranks' times (ms); identity on one rank."""
    if world <= 1:
        return t_ms
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_ms], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def replica_throughput(world, n_elem, steps, t_ms):
    """Whole-job elements/s: every rank processed n_elem elements per step."""
    return world * n_elem * steps / (t_ms * 1e-3)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2608_27863_gb300 import build as B
    from paper_2608_27863_gb300 import hdg as H

    cpu = None
    pool = None
    ncores = os.cpu_count() or 1
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = oracle_pool(args.workload, ncores)      # before the first GPU call

    torch.cuda.set_device(local_rank)
    B.build()
    peaks, _ = H.hdg_measure_peaks()           # hand-written pipe probes on this GPU (untimed)
    wl = WORKLOADS[args.workload]
    mixed_only = wl.get("mixed_only", False)
    P = make_problem(args.workload)
    m = P.mesh
    tags = m.bnd_tag if np.any(m.bnd_tag) else None
    h = H.hdg_create(m.dim, m.vert_xyz, m.elem_vert, m.periodic_map, tags, P.p, P.gamma, P.re, P.pr, P.mach)
    H.hdg_set_params(h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s)
    if tags is not None and np.any(tags == 1):
        H.hdg_set_bc_state(h, 1, P.ubc)
    if tags is not None and np.any(tags == 3):
        H.hdg_set_bc_state(h, 3, np.array([P.twall]))
    stream = torch.cuda.current_stream()
    H.hdg_set_stream(h, stream.cuda_stream)
    dev = torch.device("cuda", local_rank)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    U, Q, UH, Us = t(P.U), t(P.Q), t(P.UH), t(P.Ustar)
    nu = None if P.nu is None else t(P.nu)
    if nu is None and "av" in wl:       # artificial viscosity of the state, computed once before timing
        nu = torch.empty(U[:, 0, :].shape, dtype=torch.float64, device=dev)
        H.hdg_av_field(h, U, Q, nu, wl["av"][0], wl["av"][1], 1.0)
    x = t(np.random.default_rng(rank).normal(size=P.UH.shape))
    y = torch.empty_like(UH)
    dQ, dU = torch.empty_like(Q), torch.empty_like(U)
    flush = torch.empty(2 * L2_BYTES // 8, dtype=torch.float64, device=dev)

    def step():
        H.hdg_linearize_condense(h, U, Q, UH, Us, nu, P.dt, P.a_ii)
        H.hdg_trace_matvec(h, x, y)
        H.hdg_recover_interior(h, y, dQ, dU)

    def set_prec(prec):
        H.hdg_set_params(h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s, precision=prec)

    def timed(nsteps, clk_index=None):
        H.hdg_profile_read(h)
        H.hdg_profile(h, True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        times = []
        with ClockSampler(local_rank if clk_index is None else clk_index) as clk:
            for _ in range(nsteps):
                flush.fill_(1.0)       # L2 flush between timed steps (not timed)
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record(stream)
                step()
                e.record(stream)
                e.synchronize()
                times.append(s.elapsed_time(e))
        torch.cuda.synchronize()
        prof = H.hdg_profile_read(h)
        H.hdg_profile(h, False)
        t_ms = max_over_ranks(sum(times), world, dev)
        if world > 1:
            dist.barrier()
        return t_ms, prof, clk.summary()

    def tune(fp64):
        # the project's autotuner picks among equivalent kernel variants on these inputs (untimed)
        if args.no_autotune or args.elim_nb or args.tuning:
            if args.elim_nb or args.tuning:      # a fixed variant (profiling runs)
                kw = dict(elim_nb=args.elim_nb or 16, elim_minb=2,
                          schur_mode=0 if fp64 else {"fp32": 0, "tf32": 1, "3xtf32": 2}[args.mixed_prec],
                          blocks_mode=1 if m.dim == 3 else 0, elim_mixed_minb=2, blocks64_mode=1)
                # "--tuning k=v,..." sets both legs; "fp64.k=v" / "mixed.k=v" one leg
                for item in (args.tuning or "").split(","):
                    if item:
                        k, v = item.split("=")
                        leg, _, key = k.rpartition(".")
                        if not leg or leg == ("fp64" if fp64 else "mixed"):
                            kw[key] = int(v)
                H.hdg_set_tuning(h, **kw)
                return dict(kw, fixed=True)
            return None
        rep = H.hdg_autotune(h, U, Q, UH, Us, nu, P.dt, P.a_ii, reps=1)
        return {k: rep[k] for k in ("elim_nb", "elim_minb", "schur_mode", "blocks_mode", "elim_mixed_minb",
                                    "blocks64_mode", "elim_mixed_split")}

    # FP64 form (the headline value); skipped when its arrays would not fit in HBM
    dgemm = fp64_peak_tflops(torch)
    tuning = {}
    if not mixed_only:
        set_prec(H.HDG_PREC_FP64)
        tuning["fp64"] = tune(True)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if H.hdg_status(h) != 0:
            raise RuntimeError("device status: " + H.hdg_last_error(h))
        t_ms, prof, clocks = timed(args.steps)

    # mixed form on the same workload and step
    mixed_prec = {"fp32": H.HDG_PREC_MIXED, "tf32": H.HDG_PREC_MIXED_TF32,
                  "3xtf32": H.HDG_PREC_MIXED_3XTF32}[args.mixed_prec]
    set_prec(mixed_prec)
    tuning["mixed"] = tune(False)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if H.hdg_status(h) != 0:
        raise RuntimeError("device status (mixed): " + H.hdg_last_error(h))
    tm_ms, prof_m, clocks_m = timed(args.steps)
    if mixed_only:
        t_ms, prof, clocks = tm_ms, prof_m, clocks_m
    else:
        set_prec(H.HDG_PREC_FP64)

    # end to end through the C-ABI from pinned host memory
    hU, hQ, hUH, hUs = (torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (P.U, P.Q, P.UH, P.Ustar))
    hdQ = torch.empty(dQ.shape, dtype=torch.float64).pin_memory()
    hdU = torch.empty(dU.shape, dtype=torch.float64).pin_memory()
    h2d = sum(a.numel() * 8 for a in (hU, hQ, hUH, hUs))
    d2h = (hdQ.numel() + hdU.numel()) * 8
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        U.copy_(hU, non_blocking=True)
        Q.copy_(hQ, non_blocking=True)
        UH.copy_(hUH, non_blocking=True)
        Us.copy_(hUs, non_blocking=True)
        step()
        hdQ.copy_(dQ, non_blocking=True)
        hdU.copy_(dU, non_blocking=True)
        e.record(stream)
        e.synchronize()
        e2e_ms += s.elapsed_time(e)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)

    check_ids, check_refs = None, None
    if pool is not None:
        n_sample = make_problem(args.workload, cpu_sample=True).mesh.n_elem if "cpu" in wl else m.n_elem
        rate, n_done, secs = oracle_rate(pool, ncores, n_sample, args.cpu_seconds, 100)
        if "cpu" not in wl and not ("av" in wl and P.nu is None):
            # the oracle's elements are this workload's (same mesh, state and viscosity field)
            check_ids = oracle_check_elements(n_elem=m.n_elem)
            check_refs = pool.map(_worker_schur, check_ids)
        pool.close()
        cpu = {"value": rate, "unit": "elements/s", "cores": ncores, "cpu_model": cpu_model(), "kind": "oracle",
               "sample": "%d seeded elements of %s in %.1f s: per-element residual, complex-step "
                         "Jacobian, dense FP64 LU of the (q,u) block and Schur complement (assembly, matvec "
                         "and recovery not included)" % (n_done, "a %d-element mesh of the same elements and physics"
                                                         % n_sample if "cpu" in wl else "the same workload", secs)}

    oracle_check = None
    if check_ids is not None:
        # per-element S^K of both forms against the oracle's condensation of the same elements (untimed)
        t_el = H.hdg_query_sizes(h)["t"]
        ts = np.full(m.n_elem, t_el, dtype=np.int64)
        offs = np.arange(m.n_elem + 1, dtype=np.int64) * t_el * t_el

        def hex_prec(prec):
            set_prec(prec)
            tn = tuning.get("fp64" if prec == H.HDG_PREC_FP64 else "mixed")
            if tn:
                H.hdg_set_tuning(h, **{k: v for k, v in tn.items() if k != "fixed"})

        run1 = lambda: H.hdg_linearize_condense(h, U, Q, UH, Us, nu, P.dt, P.a_ii)
        precs = {"mixed": (mixed_prec, hex_prec, run1)}
        if not mixed_only:
            precs["fp64"] = (H.HDG_PREC_FP64, hex_prec, run1)
        oracle_check = element_block_errors(H, h, torch, check_ids, offs, ts, check_refs, precs)
        oracle_check = {"what": "relative Frobenius error of the per-element Schur complement S^K against the "
                                "FP64 CPU oracle's condensation of the same element",
                        "elements": check_ids, **oracle_check}
        set_prec(H.HDG_PREC_FP64)

    # mixed vs FP64 at tolerance: Newton on the stage equations to ||F||_2 <= 1e-8 (FP64 residual)
    newton = {}
    if not args.no_newton and not mixed_only:
        for name, prec in (("fp64", H.HDG_PREC_FP64), ("mixed", mixed_prec)):
            set_prec(prec)
            U2, Q2, UH2 = U.clone(), Q.clone(), UH.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            nit, git, hist = H.hdg_newton(h, U2, Q2, UH2, Us, nu, P.dt, P.a_ii, tol=1e-8, max_newton=12,
                                          restart=40, max_gmres=600, gmres_rtol=1e-9, raise_on_noconv=False)
            torch.cuda.synchronize()
            newton[name] = {"seconds": time.perf_counter() - t0, "newton_iters": nit, "gmres_iters": git,
                            "residual_history": [float(v) for v in hist]}
            newton[name + "_state"] = (U2, UH2)
        du = float(torch.linalg.norm(newton["mixed_state"][0] - newton["fp64_state"][0]) /
                   torch.linalg.norm(newton["fp64_state"][0]))
        duh = float(torch.linalg.norm(newton["mixed_state"][1] - newton["fp64_state"][1]) /
                    torch.linalg.norm(newton["fp64_state"][1]))
        del newton["mixed_state"], newton["fp64_state"]
        newton["tol"] = 1e-8
        newton["state_rel_diff_U"] = du
        newton["state_rel_diff_UH"] = duh
        newton["speedup"] = newton["fp64"]["seconds"] / newton["mixed"]["seconds"]
        set_prec(H.HDG_PREC_FP64)

    E = m.n_elem
    if mixed_only:
        out = mixed_only_line(args, world, E, P, m, h, tm_ms, prof_m, clocks_m, e2e_ms, h2d, d2h, dgemm)
        out["tuning"] = tuning
        if cpu is not None:
            out["cpu_baseline"] = cpu
        H.hdg_destroy(h)
        return out
    t64 = tuning.get("fp64") or {}
    oz = t64.get("schur_mode", 0) == 3          # FP64 Schur product on the tensor cores
    fl = flop_counts(m.dim, P.p, sum_factorised=t64.get("blocks64_mode", 1) == 1, tc_schur=oz)
    nb_used = t64.get("elim_nb", args.elim_nb or 16)
    kern = {}
    for k, (ms, n) in prof.items():
        if n:
            kern[k] = {"ms_per_step": ms / args.steps, "launches_per_step": n / args.steps}
    kern["elim"]["tflops"] = fl["elim"] * E / (prof["elim"][0] / args.steps) / 1e9
    kern["blocks"]["tflops"] = fl["blocks"] * E / (prof["blocks"][0] / args.steps) / 1e9
    if oz and prof["schur"][1]:
        # FP64-equivalent rate of the emulated product, and the BF16 tensor work it executes
        kern["schur"]["fp64_equivalent_tflops"] = fl["schur"] * E / (prof["schur"][0] / args.steps) / 1e9
        kern["schur"]["bf16_tflops_executed"] = fl["schur_bf16"] * E / (prof["schur"][0] / args.steps) / 1e9
        kern["schur"]["bf16_frac_of_probe"] = kern["schur"]["bf16_tflops_executed"] / peaks["bf16_tcgen05"]
    dom = max(("elim", "blocks"), key=lambda k: prof[k][0])
    sf64 = t64.get("blocks64_mode", 1) == 1
    dom_name = dom + ("_sf" if dom == "blocks" and sf64 else "")
    traffic_key = (dom_name, m.dim, P.p, nb_used if dom == "elim" and not oz else 0)
    dom_kernels = {"elim": "k_elim", "blocks_sf": "k_blocks_sf + k_blocks (face terms)", "blocks": "k_blocks"}
    avg_launch_ms = prof[dom][0] / max(prof[dom][1], 1)
    per_launch_elems = E / max(prof[dom][1] / args.steps, 1)
    achieved = fl[dom] * per_launch_elems / (avg_launch_ms * 1e-3) / 1e12
    smmax = clocks.get("sm_max_mhz") or 2070.0
    peak = fp64_peak_derived(smmax)
    launches = sum(n for _, n in prof.values()) / args.steps
    value = replica_throughput(world, E, args.steps, t_ms)
    mixed = {"value": replica_throughput(world, E, args.steps, tm_ms), "unit": "elements/s", "ms_per_step": tm_ms / args.steps,
             "speedup_vs_fp64_step": t_ms / tm_ms,
             "kernels": {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
                         for k, v in prof_m.items() if v[1]},
             "dtype": "fp64 residual, interior LU (pivoting) and Arnoldi; fp32 Jacobian terms and blocks; Schur "
                      "product %s" % {"fp32": "fp32 SIMT", "tf32": "TF32 tensor cores (tcgen05)",
                                      "3xtf32": "3xTF32 tensor cores (tcgen05)"}[args.mixed_prec],
             "clocks": clocks_m}
    lu_flops = sum(2 * (C_nu - k - 1) * (C_nu - k) + (C_nu - k - 1) for C_nu in [(m.dim + 2) * (P.p + 1) ** m.dim]
                   for k in range(C_nu))
    mixed["fp64_lu_tflops"] = lu_flops * E / (prof_m["elim"][0] / args.steps) / 1e9
    if newton:
        mixed["newton"] = newton
    out = {
        "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "elements_per_gpu": E, "degree": P.p, "dim": m.dim,
                   "faces": H.hdg_query_sizes(h)["n_faces"], "parallelism": "replicas" if world > 1 else "single",
                   "precision": "fp64", "l2": "flushed between timed steps (256 MiB write)"},
        "roofline": {"bound": "alu", "kernel": dom_kernels[dom_name], "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": (DRAM_BYTES_PER_ELEMENT[traffic_key] * per_launch_elems
                                 if traffic_key in DRAM_BYTES_PER_ELEMENT else None),
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one %s launch on the "
                                       "8^3 case, per element, times the elements of one launch" % dom_kernels[dom_name],
                     "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x %.0f MHz (derived); cuBLAS DGEMM "
                                    "measured in this run: %.3f TFLOP/s" % (smmax, dgemm),
                     "peak_measured": peaks["fp64_fma"], "frac_of_measured": achieved / peaks["fp64_fma"],
                     "peak_measured_source": "DFMA-chain probe (hdg_measure_peaks) in this run",
                     "flops_per_element": fl[dom]},
        "gflops_total": fl["total"] * E * args.steps / (t_ms * 1e-3) / 1e9,
        "kernels": kern,
        "recover_roofline": recover_roofline("k_recover", hex_recover_bytes(m.dim, P.p, E), prof["recover"]),
        "mixed": mixed,
        "e2e": {"value": replica_throughput(world, E, args.steps, e2e_ms), "unit": "elements/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
        "tuning": tuning,
        "peaks_measured_tflops": peaks,
    }
    if oracle_check is not None:
        out["oracle_check"] = oracle_check
        mixed["block_err_vs_oracle"] = oracle_check["mixed"]["max_rel_err"]
    if cpu is not None:
        out["cpu_baseline"] = cpu
    H.hdg_destroy(h)
    return out


def fp64_lu_flops(d, p):
    """FP64 flops of the interior LU with pivoting in the mixed elimination (per element)."""
    nu = (d + 2) * (p + 1) ** d
    return sum(2 * (nu - k - 1) * (nu - k) + (nu - k - 1) for k in range(nu))


def mixed_only_line(args, world, E, P, m, h, tm_ms, prof_m, clocks_m, e2e_ms, h2d, d2h, dgemm):
    """JSON line of a workload timed in the mixed form only; the roofline is that of
    the mixed elimination's FP64 interior LU (its dominant kernel)."""
    from paper_2608_27863_gb300 import hdg as H
    lu = fp64_lu_flops(m.dim, P.p)
    ms, n = prof_m["elim"]
    per_launch = E / max(n / args.steps, 1)
    achieved = lu * per_launch / ((ms / max(n, 1)) * 1e-3) / 1e12
    smmax = clocks_m.get("sm_max_mhz") or 2070.0
    peak = fp64_peak_derived(smmax)
    sizes = H.hdg_query_sizes(h)
    kern = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
            for k, v in prof_m.items() if v[1]}
    return {
        "metric": METRIC, "value": replica_throughput(world, E, args.steps, tm_ms), "unit": "elements/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tm_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "mixed", "data": "synthetic",
        "config": {"workload": args.workload, "elements_per_gpu": E, "degree": P.p, "dim": m.dim,
                   "faces": sizes["n_faces"], "parallelism": "replicas" if world > 1 else "single",
                   "precision": "mixed (fp64 residual and interior LU; fp32 Jacobians and trace blocks; Schur "
                                "product %s)" % args.mixed_prec,
                   "device_bytes": sizes["device_bytes"],
                   "l2": "flushed between timed steps (256 MiB write); inputs far above L2"},
        "roofline": {"bound": "alu", "kernel": "k_elim_mixed", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                     "flops_per_element": lu,
                     "peak_source": "FP64 pipe: 152 SMs x 2 DFMA/clk x 2 flop x %.0f MHz (derived); cuBLAS DGEMM "
                                    "measured in this run: %.3f TFLOP/s; flops: the FP64 interior LU only" %
                                    (smmax, dgemm)},
        "kernels": kern,
        "e2e": {"value": replica_throughput(world, E, args.steps, e2e_ms), "unit": "elements/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": sum(n for _, n in prof_m.values()) / args.steps,
        "clocks": clocks_m,
    }


def run_reference(args, rank, world):
    """The FP64 CPU oracle as it stands, on the host cores, same workload and metric."""
    if rank != 0:
        return None
    ncores = os.cpu_count() or 1
    if WORKLOADS[args.workload].get("kind") == "tet":
        from synth import tetmesh as tm
        n_elem = tm.config4_mesh(**WORKLOADS[args.workload]["kw"]).n_elem
        degree = "1..4"
    else:
        P = make_problem(args.workload, cpu_sample=True)      # the elements the oracle samples from
        n_elem, degree = P.mesh.n_elem, P.p
    pool = oracle_pool(args.workload, ncores)
    for w in range(args.warmup):
        oracle_rate(pool, ncores, n_elem, 0.0, 500 + w)
    tot_e, tot_s = 0, 0.0
    for k in range(args.steps):
        _, n, s = oracle_rate(pool, ncores, n_elem, 0.0, 900 + k)
        tot_e += n
        tot_s += s
    pool.close()
    rate = tot_e / tot_s
    return {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "elements/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "elements_per_gpu": n_elem, "degree": degree},
        "cpu_baseline": {"value": rate, "unit": "elements/s", "cores": ncores, "cpu_model": cpu_model(), "kind": "oracle",
                         "sample": "each step condenses %d seeded elements (one per core) of the workload" % ncores},
        "e2e": {"value": rate, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-newton", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="tetrahedral workloads: time the FP64 form only")
    ap.add_argument("--dirk", action="store_true",
                    help="tetrahedral workloads: also time one graph-captured SDIRK3 step (3 stages x "
                         "--dirk-newton Newton iterations x GMRES(--dirk-m))")
    ap.add_argument("--mixed-prec", choices=["fp32", "tf32", "3xtf32"], default="3xtf32")
    ap.add_argument("--precond", choices=["schwarz", "bj"], default="schwarz",
                    help="tetrahedral workloads: preconditioner of the Newton comparison's GMRES")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--dirk-newton", type=int, default=5, help="Newton iterations per stage of the --dirk step")
    ap.add_argument("--dirk-m", type=int, default=100, help="GMRES iterations per Newton step of the --dirk step")
    ap.add_argument("--elim-nb", type=int, choices=[8, 16], default=None,
                    help="fix the FP64 elimination panel width instead of autotuning (profiling runs)")
    ap.add_argument("--tuning", default=None,
                    help="fixed kernel variants instead of autotuning, e.g. elim_nb=8,elim_minb=1,"
                         "blocks64_mode=1,blocks_mode=1,elim_mixed_minb=3,fp64.schur_mode=3 (profiling runs; "
                         "a 'fp64.' or 'mixed.' prefix applies an item to one leg)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        out = (run_tet if WORKLOADS[args.workload].get("kind") == "tet" else run_ours)(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
