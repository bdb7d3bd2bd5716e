"""Shared test helpers: run the library on a synth.Problem and read results back."""
from __future__ import annotations

import numpy as np

import paper_2608_27863_gb300.hdg as H


def create(P, host_only=False):
    m = P.mesh
    h = H.hdg_create(m.dim, m.vert_xyz, m.elem_vert, m.periodic_map,
                     m.bnd_tag if np.any(m.bnd_tag) else None, P.p, P.gamma, P.re, P.pr, P.mach,
                     host_only=host_only)
    if not host_only:
        H.hdg_set_params(h, tau=P.tau, visc_law=P.visc_law, suth_c1=P.suth_c1, suth_s=P.suth_s,
                         tau_mode=getattr(P, "tau_mode", 0))
        if np.any(m.bnd_tag == 1):
            ubc = np.asarray(P.ubc, dtype=np.float64)
            if ubc.ndim == 1:
                H.hdg_set_bc_state(h, 1, ubc)
            else:
                import torch
                H.hdg_set_bc_field(h, torch.from_numpy(np.ascontiguousarray(ubc)).cuda())
        if np.any(m.bnd_tag == 3):
            H.hdg_set_bc_state(h, 3, np.array([P.twall]))
    return h


class GpuRun:
    """One linearization of problem P on the GPU, with host copies of the results."""

    def __init__(self, P, h=None):
        import torch
        self.torch = torch
        self.P = P
        self.h = h if h is not None else create(P)
        dev = torch.device("cuda")
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
        self.U, self.Q, self.UH, self.Ustar = t(P.U), t(P.Q), t(P.UH), t(P.Ustar)
        self.nu = None if P.nu is None else t(P.nu)
        self.sizes = H.hdg_query_sizes(self.h)
        H.hdg_set_stream(self.h, torch.cuda.current_stream().cuda_stream)

    def linearize(self):
        H.hdg_linearize_condense(self.h, self.U, self.Q, self.UH, self.Ustar, self.nu, self.P.dt, self.P.a_ii)
        return self

    def blocks(self):
        """BSR values as [nnzb][block][block], semantic row-major (r, c)."""
        s = self.sizes
        v = self.torch.empty(s["nnzb"] * s["block"] * s["block"], dtype=self.torch.float64, device="cuda")
        H.hdg_get_blocks(self.h, v)
        self.torch.cuda.synchronize()
        return v.cpu().numpy().reshape(s["nnzb"], s["block"], s["block"]).transpose(0, 2, 1)

    def rhs(self):
        g = self.torch.empty_like(self.UH)
        H.hdg_trace_rhs(self.h, g)
        self.torch.cuda.synchronize()
        return g.cpu().numpy()

    def matvec(self, x):
        xd = self.torch.from_numpy(np.ascontiguousarray(x)).cuda()
        y = self.torch.empty_like(xd)
        H.hdg_trace_matvec(self.h, xd, y)
        self.torch.cuda.synchronize()
        return y.cpu().numpy()

    def recover(self, dUH):
        d = self.torch.from_numpy(np.ascontiguousarray(dUH)).cuda()
        dQ = self.torch.empty_like(self.Q)
        dU = self.torch.empty_like(self.U)
        H.hdg_recover_interior(self.h, d, dQ, dU)
        self.torch.cuda.synchronize()
        return dQ.cpu().numpy(), dU.cpu().numpy()

    def close(self):
        H.hdg_destroy(self.h)


def block_rel_errors(gpu_vals, orc_vals: dict):
    """Relative Frobenius error of each compared block.  A block that is zero
    in the oracle (the off-diagonal blocks of a boundary face whose trace rows
    do not depend on the interior) is measured against the mean block norm."""
    scale = np.mean([np.linalg.norm(r) for r in orc_vals.values()])
    out = {}
    for b, ref in orc_vals.items():
        nr = np.linalg.norm(ref)
        out[b] = np.linalg.norm(gpu_vals[b] - ref) / (nr if nr > 0 else scale)
    return out
