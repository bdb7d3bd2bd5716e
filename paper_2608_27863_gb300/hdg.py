"""ctypes binding of libhdg.so: the C-ABI of ``include/hdg.h`` under the same names.

Argument marshalling only: device arrays are torch CUDA tensors (float64,
contiguous) passed by ``data_ptr()``; every step of the computation runs in the
library's kernels.  A missing library raises ``HDGError`` -- there is no
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhdg.so")

HDG_OK = 0
HDG_EINVAL = -1
HDG_ENOMEM = -2
HDG_ECUDA = -3
HDG_ESINGULAR = -4
HDG_ENONFINITE = -5
HDG_ENOCONV = -6
HDG_EUNSUPPORTED = -7
HDG_QUAD = 1
HDG_HEX = 2
HDG_TET = 3
HDG_PREC_FP64 = 0
HDG_PREC_MIXED = 1
HDG_PREC_MIXED_TF32 = 2
HDG_PREC_MIXED_3XTF32 = 3

EXPORTS = [
    "hdg_create", "hdg_create_host", "hdg_destroy", "hdg_last_error", "hdg_set_params", "hdg_set_stream",
    "hdg_query_sizes", "hdg_get_connectivity", "hdg_linearize_condense", "hdg_trace_matvec",
    "hdg_trace_rhs", "hdg_recover_interior", "hdg_get_blocks", "hdg_status", "hdg_profile",
    "hdg_profile_read", "hdg_linearize_condense_static", "hdg_residual", "hdg_update_state",
    "hdg_blockjacobi_setup", "hdg_blockjacobi_apply", "hdg_gmres", "hdg_newton", "hdg_set_bc_state",
    "hdg_newton_fixed", "hdg_dirk_step", "hdg_lift_gradient", "hdg_set_preconditioner", "hdg_schwarz_setup",
    "hdg_schwarz_apply", "hdg_rb_setup", "hdg_rb_push", "hdg_rb_guess", "hdg_av_field", "hdg_tgv_diagnostics",
    "hdg_autotune", "hdg_set_tuning", "hdg_set_bc_field", "hdg_reserve", "hdg_create_tet", "hdg_create_tet_host",
    "hdg_tet_query", "hdg_tet_layout", "hdg_tet_ref_tables", "hdg_tri_ref_tables", "hdg_partition",
    "hdg_part_layout", "hdg_sdirk3_tableau", "hdg_measure_peaks", "hdg_set_element_block_output",
]
KERNEL_CLASSES = ["point", "blocks", "elim", "assemble", "matvec", "recover", "schur"]


class HDGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libhdg error %d: %s" % (code, msg))
        self.code = code


class hdg_mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("elem_type", ctypes.c_int32), ("n_elem", ctypes.c_int64),
                ("n_vert", ctypes.c_int64), ("vert_xyz", ctypes.c_void_p), ("elem_vert", ctypes.c_void_p),
                ("periodic_map", ctypes.c_void_p), ("bnd_tag", ctypes.c_void_p)]


class hdg_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("visc_law", ctypes.c_int32), ("suth_c1", ctypes.c_double),
                ("suth_s", ctypes.c_double), ("precision", ctypes.c_int32), ("tau_mode", ctypes.c_int32)]


class hdg_sizes(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("dim", "p", "m", "Np", "Nq", "nf", "Nfp", "Nfq", "n_u", "n_q", "t",
                                               "block")] + \
               [(n, ctypes.c_int64) for n in ("n_elem", "n_faces", "nnzb", "device_bytes")]


class hdg_tet_mesh(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int64), ("n_vert", ctypes.c_int64), ("vert_xyz", ctypes.c_void_p),
                ("elem_vert", ctypes.c_void_p), ("periodic_map", ctypes.c_void_p), ("bnd_tag", ctypes.c_void_p),
                ("elem_p", ctypes.c_void_p), ("geo", ctypes.c_void_p)]


class hdg_tet_sizes(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("n_elem", "n_faces", "nnzb", "n_u", "n_trace", "n_vals", "n_curved",
                                               "device_bytes")]


class hdg_part_sizes(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int64), ("n_interior_elem", ctypes.c_int64), ("n_faces", ctypes.c_int64),
                ("n_interface_faces", ctypes.c_int64), ("n_halo_faces", ctypes.c_int64)]


_lib = None


def lib():
    """Load libhdg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise HDGError(HDG_EINVAL, "libhdg.so not found at %s; build it with "
                                   "paper_2608_27863_gb300.build.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "hdg_create": [ctypes.POINTER(vp), ctypes.POINTER(hdg_mesh), i32, dbl, dbl, dbl, dbl],
        "hdg_create_host": [ctypes.POINTER(vp), ctypes.POINTER(hdg_mesh), i32, dbl, dbl, dbl, dbl],
        "hdg_destroy": [vp],
        "hdg_set_params": [vp, ctypes.POINTER(hdg_params)],
        "hdg_set_stream": [vp, vp],
        "hdg_set_bc_state": [vp, i32, vp],
        "hdg_query_sizes": [vp, ctypes.POINTER(hdg_sizes)],
        "hdg_get_connectivity": [vp] * 7,
        "hdg_linearize_condense": [vp, vp, vp, vp, vp, vp, dbl, dbl, vp],
        "hdg_trace_matvec": [vp, vp, vp],
        "hdg_trace_rhs": [vp, vp],
        "hdg_recover_interior": [vp, vp, vp, vp],
        "hdg_get_blocks": [vp, vp],
        "hdg_status": [vp],
        "hdg_profile": [vp, i32],
        "hdg_profile_read": [vp, vp, vp],
        "hdg_linearize_condense_static": [vp, vp, vp, vp, vp, vp, dbl, dbl],
        "hdg_residual": [vp, vp, vp, vp, vp, vp, dbl, dbl, vp, vp, vp, vp],
        "hdg_update_state": [vp, vp, vp, vp, vp, vp, vp, dbl],
        "hdg_blockjacobi_setup": [vp],
        "hdg_blockjacobi_apply": [vp, vp, vp],
        "hdg_gmres": [vp, vp, vp, i32, i32, dbl, i32, vp, vp],
        "hdg_newton": [vp, vp, vp, vp, vp, vp, dbl, dbl, dbl, i32, i32, i32, dbl, vp, vp, vp],
        "hdg_lift_gradient": [vp, vp, vp, vp],
        "hdg_set_preconditioner": [vp, i32],
        "hdg_schwarz_setup": [vp],
        "hdg_schwarz_apply": [vp, vp, vp],
        "hdg_rb_setup": [vp, i32],
        "hdg_autotune": [vp, vp, vp, vp, vp, vp, dbl, dbl, i32, vp],
        "hdg_set_tuning": [vp, vp],
        "hdg_set_bc_field": [vp, vp],
        "hdg_reserve": [vp, i32],
        "hdg_av_field": [vp, vp, vp, dbl, dbl, dbl, vp],
        "hdg_tgv_diagnostics": [vp, vp, vp, vp],
        "hdg_rb_push": [vp, vp],
        "hdg_rb_guess": [vp, vp, vp],
        "hdg_newton_fixed": [vp, vp, vp, vp, vp, vp, dbl, dbl, i32, i32, i32, vp],
        "hdg_dirk_step": [vp, vp, vp, vp, vp, dbl, i32, vp, vp, i32, i32, i32, vp],
        "hdg_sdirk3_tableau": [vp, vp],
        "hdg_measure_peaks": [vp, vp],
        "hdg_set_element_block_output": [vp, vp],
        "hdg_create_tet": [ctypes.POINTER(vp), ctypes.POINTER(hdg_tet_mesh), dbl, dbl, dbl, dbl],
        "hdg_create_tet_host": [ctypes.POINTER(vp), ctypes.POINTER(hdg_tet_mesh), dbl, dbl, dbl, dbl],
        "hdg_tet_query": [vp, ctypes.POINTER(hdg_tet_sizes)],
        "hdg_tet_layout": [vp] * 10,
        "hdg_tet_ref_tables": [i32, vp, vp, vp, vp],
        "hdg_tri_ref_tables": [i32, vp, vp, vp],
        "hdg_partition": [vp, i32, vp],
        "hdg_part_layout": [vp, vp, i32, ctypes.POINTER(hdg_part_sizes)] + [vp] * 6,
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.hdg_last_error.argtypes = [vp]
    L.hdg_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(h, rc):
    if rc != HDG_OK:
        msg = lib().hdg_last_error(h).decode() if h else "error"
        raise HDGError(rc, msg)


def _ptr(t):
    """Device pointer of a torch CUDA float64 tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise HDGError(HDG_EINVAL, "arguments must be contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


class _MeshArgs:
    """Keeps the host arrays of an hdg_mesh alive for the duration of a call."""

    def __init__(self, dim, vert_xyz, elem_vert, periodic_map=None, bnd_tag=None):
        self.vert = np.ascontiguousarray(vert_xyz, dtype=np.float64)
        self.ev = np.ascontiguousarray(elem_vert, dtype=np.int64)
        self.pm = None if periodic_map is None else np.ascontiguousarray(periodic_map, dtype=np.int64)
        self.bt = None if bnd_tag is None else np.ascontiguousarray(bnd_tag, dtype=np.int32)
        self.s = hdg_mesh(dim, HDG_QUAD if dim == 2 else HDG_HEX, self.ev.shape[0], self.vert.shape[0],
                          self.vert.ctypes.data, self.ev.ctypes.data,
                          None if self.pm is None else self.pm.ctypes.data,
                          None if self.bt is None else self.bt.ctypes.data)


def hdg_create(dim, vert_xyz, elem_vert, periodic_map, bnd_tag, p, gamma, Re, Pr, Mach, host_only=False):
    """Create a handle; returns it as a ctypes void pointer."""
    m = _MeshArgs(dim, vert_xyz, elem_vert, periodic_map, bnd_tag)
    h = ctypes.c_void_p()
    fn = lib().hdg_create_host if host_only else lib().hdg_create
    rc = fn(ctypes.byref(h), ctypes.byref(m.s), p, gamma, Re, Pr, Mach)
    if rc != HDG_OK:
        msg = lib().hdg_last_error(h).decode() if h else "error"
        lib().hdg_destroy(h)
        raise HDGError(rc, msg)
    return h


def hdg_create_host(dim, vert_xyz, elem_vert, periodic_map, bnd_tag, p, gamma, Re, Pr, Mach):
    return hdg_create(dim, vert_xyz, elem_vert, periodic_map, bnd_tag, p, gamma, Re, Pr, Mach, host_only=True)


def hdg_destroy(h):
    lib().hdg_destroy(h)


def hdg_last_error(h):
    return lib().hdg_last_error(h).decode()


def hdg_set_params(h, tau=5.0, visc_law=0, suth_c1=1.4042, suth_s=0.40417, precision=HDG_PREC_FP64, tau_mode=0):
    prm = hdg_params(tau, visc_law, suth_c1, suth_s, precision, tau_mode)
    _check(h, lib().hdg_set_params(h, ctypes.byref(prm)))


def hdg_set_bc_state(h, tag, ub):
    ub = np.ascontiguousarray(ub, dtype=np.float64)
    _check(h, lib().hdg_set_bc_state(h, int(tag), ub.ctypes.data))


def hdg_set_stream(h, stream_handle):
    _check(h, lib().hdg_set_stream(h, ctypes.c_void_p(stream_handle)))


def hdg_query_sizes(h):
    s = hdg_sizes()
    _check(h, lib().hdg_query_sizes(h, ctypes.byref(s)))
    return {n: getattr(s, n) for n, _ in hdg_sizes._fields_}


def hdg_get_connectivity(h):
    s = hdg_query_sizes(h)
    E, F, nf, Nfp, nnzb = s["n_elem"], s["n_faces"], s["nf"], s["Nfp"], s["nnzb"]
    out = {"f2e": np.zeros((F, 2), np.int32), "f2lf": np.zeros((F, 2), np.int32),
           "e2f": np.zeros((E, nf), np.int32), "perm": np.zeros((E, nf, Nfp), np.int32),
           "rowptr": np.zeros(F + 1, np.int32), "col": np.zeros(nnzb, np.int32)}
    _check(h, lib().hdg_get_connectivity(h, *[out[k].ctypes.data for k in
                                              ("f2e", "f2lf", "e2f", "perm", "rowptr", "col")]))
    return out


def hdg_linearize_condense(h, U, Q, UH, Ustar, nu, dt, a_ii, res_norm=False):
    """Linearize + condense at W = (Q, U, UH).  With res_norm=True the call also
    returns the FP64 ||F(W)||_2 that the library evaluates (and synchronises)."""
    out = ctypes.c_double(0.0)
    _check(h, lib().hdg_linearize_condense(h, _ptr(U), _ptr(Q), _ptr(UH), _ptr(Ustar), _ptr(nu),
                                           float(dt), float(a_ii), ctypes.byref(out) if res_norm else None))
    return out.value if res_norm else None


def hdg_linearize_condense_static(h, U, Q, UH, Ustar, nu, dt, a_ii):
    """Allocation-free variant: scratch from the library's static device array."""
    _check(h, lib().hdg_linearize_condense_static(h, _ptr(U), _ptr(Q), _ptr(UH), _ptr(Ustar), _ptr(nu),
                                                  float(dt), float(a_ii)))


def hdg_trace_matvec(h, x, y):
    _check(h, lib().hdg_trace_matvec(h, _ptr(x), _ptr(y)))


def hdg_trace_rhs(h, g):
    _check(h, lib().hdg_trace_rhs(h, _ptr(g)))


def hdg_recover_interior(h, dUH, dQ, dU):
    _check(h, lib().hdg_recover_interior(h, _ptr(dUH), _ptr(dQ), _ptr(dU)))


def hdg_get_blocks(h, vals):
    _check(h, lib().hdg_get_blocks(h, _ptr(vals)))


def hdg_set_element_block_output(h, SK):
    """Later linearizations also write every element's S^K to SK (device tensor), or None to stop."""
    _check(h, lib().hdg_set_element_block_output(h, _ptr(SK)))


def hdg_status(h):
    return lib().hdg_status(h)


def hdg_profile(h, enable=True):
    _check(h, lib().hdg_profile(h, 1 if enable else 0))


def hdg_profile_read(h):
    """{kernel class: (milliseconds, launches)} accumulated since the last read."""
    ms = np.zeros(len(KERNEL_CLASSES), np.float64)
    n = np.zeros(len(KERNEL_CLASSES), np.int64)
    _check(h, lib().hdg_profile_read(h, ms.ctypes.data, n.ctypes.data))
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_CLASSES)}


def hdg_residual(h, U, Q, UH, Ustar, nu, dt, a_ii, Rq=None, Ru=None, Ruh=None):
    """FP64 stage residual; returns (||F||, ||(R_q, R_u)||, ||R_uhat||)."""
    norms = np.zeros(3, np.float64)
    _check(h, lib().hdg_residual(h, _ptr(U), _ptr(Q), _ptr(UH), _ptr(Ustar), _ptr(nu), float(dt), float(a_ii),
                                 _ptr(Rq), _ptr(Ru), _ptr(Ruh), norms.ctypes.data))
    return tuple(float(v) for v in norms)


def hdg_update_state(h, U, Q, UH, dU, dQ, dUH, alpha):
    _check(h, lib().hdg_update_state(h, _ptr(U), _ptr(Q), _ptr(UH), _ptr(dU), _ptr(dQ), _ptr(dUH), float(alpha)))


def hdg_blockjacobi_setup(h):
    _check(h, lib().hdg_blockjacobi_setup(h))


def hdg_blockjacobi_apply(h, x, y):
    _check(h, lib().hdg_blockjacobi_apply(h, _ptr(x), _ptr(y)))


def hdg_gmres(h, b, x, restart=30, max_iter=300, rtol=1e-10, precond=True, raise_on_noconv=True):
    """GMRES on S x = b; returns (iterations, relative preconditioned residual)."""
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    rc = lib().hdg_gmres(h, _ptr(b), _ptr(x), int(restart), int(max_iter), float(rtol), 1 if precond else 0,
                         ctypes.byref(it), ctypes.byref(rel))
    if rc != HDG_OK and (raise_on_noconv or rc != HDG_ENOCONV):
        _check(h, rc)
    return it.value, rel.value


def hdg_newton(h, U, Q, UH, Ustar, nu, dt, a_ii, tol=1e-8, max_newton=10, restart=40, max_gmres=400,
               gmres_rtol=1e-10, raise_on_noconv=True):
    """Newton on the stage equations; returns (newton iterations, gmres iterations, residual history)."""
    hist = np.zeros(max_newton + 1, np.float64)
    nit = ctypes.c_int(0)
    git = ctypes.c_int(0)
    rc = lib().hdg_newton(h, _ptr(U), _ptr(Q), _ptr(UH), _ptr(Ustar), _ptr(nu), float(dt), float(a_ii),
                          float(tol), int(max_newton), int(restart), int(max_gmres), float(gmres_rtol),
                          hist.ctypes.data, ctypes.byref(nit), ctypes.byref(git))
    if rc != HDG_OK and (raise_on_noconv or rc != HDG_ENOCONV):
        _check(h, rc)
    return nit.value, git.value, hist[:nit.value + 1].copy()


def hdg_newton_fixed(h, U, Q, UH, Ustar, nu, dt, a_ii, n_newton=4, m=30, use_graph=True):
    """n_newton synchronisation-free Newton iterations; returns the residual history."""
    hist = np.zeros(n_newton + 1, np.float64)
    _check(h, lib().hdg_newton_fixed(h, _ptr(U), _ptr(Q), _ptr(UH), _ptr(Ustar), _ptr(nu), float(dt), float(a_ii),
                                     int(n_newton), int(m), 1 if use_graph else 0, hist.ctypes.data))
    return hist


PEAK_NAMES = ["fp64_fma", "fp64_mma", "fp32_fma", "tf32_tcgen05", "bf16_tcgen05", "int8_mma_sync"]


def hdg_measure_peaks():
    """Measured peak rates of the current device (TFLOP/s; TOP/s for INT8) and launch times."""
    t = np.zeros(6, np.float64)
    ms = np.zeros(6, np.float64)
    _check(None, lib().hdg_measure_peaks(t.ctypes.data, ms.ctypes.data))
    return {n: float(v) for n, v in zip(PEAK_NAMES, t)}, {n: float(v) for n, v in zip(PEAK_NAMES, ms)}


def sdirk3_tableau():
    """Alexander's SDIRK3 (Butcher matrix [3][3], weights [3]) as the library defines it."""
    A = np.zeros((3, 3), np.float64)
    b = np.zeros(3, np.float64)
    _check(None, lib().hdg_sdirk3_tableau(A.ctypes.data, b.ctypes.data))
    return A, b


def hdg_dirk_step(h, U, Q, UH, nu, dt, A=None, b=None, n_newton=4, m=30, use_graph=True):
    """One DIRK step in place on (U, Q, UH); returns the residual history per stage.
    A = b = None passes a NULL tableau: the library's SDIRK3."""
    if A is None and b is None:
        s, pa, pb = 3, None, None
    else:
        A = np.ascontiguousarray(A, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        s, pa, pb = A.shape[0], A.ctypes.data, b.ctypes.data
    hist = np.zeros(s * (n_newton + 1), np.float64)
    _check(h, lib().hdg_dirk_step(h, _ptr(U), _ptr(Q), _ptr(UH), _ptr(nu), float(dt), int(s), pa, pb,
                                  int(n_newton), int(m), 1 if use_graph else 0, hist.ctypes.data))
    return hist.reshape(s, n_newton + 1)


def hdg_lift_gradient(h, U, UH, Q):
    """Q <- the lifted gradient of (U, UH) (device arrays)."""
    _check(h, lib().hdg_lift_gradient(h, _ptr(U), _ptr(UH), _ptr(Q)))


HDG_PC_BLOCKJACOBI = 1
HDG_PC_SCHWARZ = 2


def hdg_set_preconditioner(h, kind):
    _check(h, lib().hdg_set_preconditioner(h, int(kind)))


def hdg_schwarz_setup(h):
    _check(h, lib().hdg_schwarz_setup(h))


def hdg_schwarz_apply(h, x, y):
    _check(h, lib().hdg_schwarz_apply(h, _ptr(x), _ptr(y)))


def hdg_rb_setup(h, nb_max):
    """Allocate and clear the reduced-basis window (nb_max = 0 disables it)."""
    _check(h, lib().hdg_rb_setup(h, int(nb_max)))


def hdg_rb_push(h, w):
    _check(h, lib().hdg_rb_push(h, _ptr(w)))


def hdg_rb_guess(h, g, x0):
    _check(h, lib().hdg_rb_guess(h, _ptr(g), _ptr(x0)))


def hdg_av_field(h, U, Q, nu, c_av, h_m, s_max=1.0):
    """nu <- smoothed artificial viscosity of the state (U, Q) (device arrays)."""
    _check(h, lib().hdg_av_field(h, _ptr(U), _ptr(Q), float(c_av), float(h_m), float(s_max), _ptr(nu)))


def hdg_tgv_diagnostics(h, U, Q):
    """(E_k, eps_S, eps_D, |Omega|) of the state (U, Q)."""
    out = np.zeros(4, np.float64)
    _check(h, lib().hdg_tgv_diagnostics(h, _ptr(U), _ptr(Q), out.ctypes.data))
    return out


class hdg_tune(ctypes.Structure):
    _fields_ = [("elim_nb", ctypes.c_int), ("elim_minb", ctypes.c_int), ("schur_mode", ctypes.c_int),
                ("blocks_mode", ctypes.c_int), ("elim_mixed_minb", ctypes.c_int), ("blocks64_mode", ctypes.c_int),
                ("elim_mixed_split", ctypes.c_int), ("n_cand", ctypes.c_int), ("cand", (ctypes.c_int * 7) * 16),
                ("ms", ctypes.c_double * 16)]


def hdg_autotune(h, U, Q, UH, Ustar, nu, dt, a_ii, reps=2):
    """Time the equivalent kernel variants on these inputs and keep the fastest; returns a dict."""
    t = hdg_tune()
    _check(h, lib().hdg_autotune(h, _ptr(U), _ptr(Q), _ptr(UH), _ptr(Ustar), _ptr(nu), float(dt), float(a_ii),
                                 int(reps), ctypes.byref(t)))
    return {"elim_nb": t.elim_nb, "elim_minb": t.elim_minb, "schur_mode": t.schur_mode,
            "blocks_mode": t.blocks_mode, "elim_mixed_minb": t.elim_mixed_minb, "blocks64_mode": t.blocks64_mode,
            "elim_mixed_split": t.elim_mixed_split,
            "candidates": [(tuple(t.cand[i]), t.ms[i]) for i in range(t.n_cand)]}


def hdg_set_tuning(h, elim_nb=16, elim_minb=2, schur_mode=0, blocks_mode=1, elim_mixed_minb=2, blocks64_mode=1,
                   elim_mixed_split=0):
    t = hdg_tune()
    t.elim_nb, t.elim_minb, t.schur_mode, t.blocks_mode = elim_nb, elim_minb, schur_mode, blocks_mode
    t.elim_mixed_minb, t.blocks64_mode, t.elim_mixed_split = elim_mixed_minb, blocks64_mode, elim_mixed_split
    _check(h, lib().hdg_set_tuning(h, ctypes.byref(t)))


def hdg_set_bc_field(h, ubf):
    """Nodal tag-1 boundary data [F][m][Nfp] (device array), or None for the constant state."""
    _check(h, lib().hdg_set_bc_field(h, _ptr(ubf)))


def hdg_reserve(h, precision=0):
    """Allocate the system storage of a precision now (it is otherwise allocated on first use)."""
    _check(h, lib().hdg_reserve(h, int(precision)))


# ----------------------------------------------------------------------------
# tetrahedral meshes of per-element degree on quadratic geometry
# ----------------------------------------------------------------------------
def hdg_create_tet(vert_xyz, elem_vert, periodic_map, bnd_tag, elem_p, geo, gamma, Re, Pr, Mach, host_only=False):
    """Handle of a tetrahedral mesh (host arrays; geo [E][10][3] or None for straight sides)."""
    keep = [np.ascontiguousarray(vert_xyz, dtype=np.float64), np.ascontiguousarray(elem_vert, dtype=np.int64),
            None if periodic_map is None else np.ascontiguousarray(periodic_map, dtype=np.int64),
            None if bnd_tag is None else np.ascontiguousarray(bnd_tag, dtype=np.int32),
            np.ascontiguousarray(elem_p, dtype=np.int32),
            None if geo is None else np.ascontiguousarray(geo, dtype=np.float64)]
    ms = hdg_tet_mesh(keep[1].shape[0], keep[0].shape[0], *[None if a is None else a.ctypes.data for a in keep])
    h = ctypes.c_void_p()
    fn = lib().hdg_create_tet_host if host_only else lib().hdg_create_tet
    rc = fn(ctypes.byref(h), ctypes.byref(ms), float(gamma), float(Re), float(Pr), float(Mach))
    if rc != HDG_OK:
        msg = lib().hdg_last_error(h).decode() if h else "error"
        if h:
            lib().hdg_destroy(h)
        raise HDGError(rc, msg)
    return h


def hdg_tet_query(h):
    s = hdg_tet_sizes()
    _check(h, lib().hdg_tet_query(h, ctypes.byref(s)))
    return {n: getattr(s, n) for n, _ in hdg_tet_sizes._fields_}


def hdg_tet_layout(h):
    s = hdg_tet_query(h)
    E, F, nnzb = s["n_elem"], s["n_faces"], s["nnzb"]
    out = {"uoff": np.zeros(E + 1, np.int64), "hoff": np.zeros(F + 1, np.int64), "face_p": np.zeros(F, np.int32),
           "f2e": np.zeros((F, 2), np.int32), "e2f": np.zeros((E, 4), np.int32),
           "frame": np.zeros((E, 4, 3), np.int32), "rowptr": np.zeros(F + 1, np.int32),
           "col": np.zeros(nnzb, np.int32), "boff": np.zeros(nnzb + 1, np.int64)}
    _check(h, lib().hdg_tet_layout(h, *[out[k].ctypes.data for k in
                                        ("uoff", "hoff", "face_p", "f2e", "e2f", "frame", "rowptr", "col", "boff")]))
    return out


def hdg_tet_ref_tables(p):
    Np, Nq = (p + 1) * (p + 2) * (p + 3) // 6, (p + 2) ** 3
    out = {"xq": np.zeros((Nq, 3)), "wq": np.zeros(Nq), "phi": np.zeros((Nq, Np)), "dphi": np.zeros((3, Nq, Np))}
    rc = lib().hdg_tet_ref_tables(int(p), *[out[k].ctypes.data for k in ("xq", "wq", "phi", "dphi")])
    if rc != HDG_OK:
        raise HDGError(rc, "hdg_tet_ref_tables")
    return out


def hdg_tri_ref_tables(p):
    Nfp, Nfq = (p + 1) * (p + 2) // 2, (p + 2) ** 2
    out = {"xs": np.zeros((Nfq, 2)), "ws": np.zeros(Nfq), "mu": np.zeros((Nfq, Nfp))}
    rc = lib().hdg_tri_ref_tables(int(p), *[out[k].ctypes.data for k in ("xs", "ws", "mu")])
    if rc != HDG_OK:
        raise HDGError(rc, "hdg_tri_ref_tables")
    return out


def hdg_partition(h, n_parts):
    """Recursive coordinate bisection of the elements into n_parts parts: elem_part [E]."""
    E = int(_n_elem(h))
    part = np.zeros(E, np.int32)
    _check(h, lib().hdg_partition(h, int(n_parts), part.ctypes.data))
    return part


def _n_elem(h):
    """Number of elements of a quad / hex or tetrahedral handle."""
    s = hdg_tet_sizes()
    if lib().hdg_tet_query(h, ctypes.byref(s)) == HDG_OK:
        return s.n_elem
    return hdg_query_sizes(h)["n_elem"]


def hdg_part_layout(h, elem_part, part):
    """Layout of one part: elements (interior first), owned faces, interface faces
    with the peer part, halo faces with their owner, and the sizes."""
    ep = np.ascontiguousarray(elem_part, dtype=np.int32)
    s = hdg_part_sizes()
    _check(h, lib().hdg_part_layout(h, ep.ctypes.data, int(part), ctypes.byref(s), *([None] * 6)))
    out = {"sizes": {n: getattr(s, n) for n, _ in hdg_part_sizes._fields_}}
    out["elems"] = np.zeros(s.n_elem, np.int64)
    out["faces"] = np.zeros(s.n_faces, np.int64)
    out["interface_faces"] = np.zeros(s.n_interface_faces, np.int64)
    out["interface_peer"] = np.zeros(s.n_interface_faces, np.int32)
    out["halo_faces"] = np.zeros(s.n_halo_faces, np.int64)
    out["halo_owner"] = np.zeros(s.n_halo_faces, np.int32)
    _check(h, lib().hdg_part_layout(h, ep.ctypes.data, int(part), ctypes.byref(s),
                                    *[out[k].ctypes.data for k in ("elems", "faces", "interface_faces",
                                                                   "interface_peer", "halo_faces", "halo_owner")]))
    return out
