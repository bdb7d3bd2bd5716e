"""The oracle's boundary forms (outflow and no-slip walls) against what the
physics fixes.

* Exact steady states give R = 0: gas at rest at the wall temperature in a box
  of isothermal walls; gas at rest at any temperature in a box of adiabatic
  walls; a uniform stream entering through a far-field face and leaving
  through an extrapolation (outflow) face.
* Conservation at a converged Newton state: with walls on every side the
  wall rows enforce zero mass flux, so sum_K 1^T M_K (U - U*) vanishes for
  density; adiabatic walls also enforce zero energy flux, so it vanishes for
  total energy too (isothermal walls conduct heat, so energy is not checked).
* Condensation + recovery equals the uncondensed global Newton solve for
  every boundary kind (brute force on 3 x 3 meshes).
"""
import numpy as np
import pytest

import synth
from oracle.dirk import newton
from oracle.hdg import Problem
from tests.test_oracle_hdg import brute_force


def with_tags(P, side_tags):
    """Set the tag of each listed box side (r, s) -> tag (sides must be non-periodic)."""
    bt = P.mesh.bnd_tag.copy()
    for (r, s), t in side_tags.items():
        col = bt[:, 2 * r + s]
        col[col != 0] = t
    P.mesh.bnd_tag = bt
    return P


def rest_state(P, T):
    """rho = 1, v = 0, T~ = T everywhere; Q = 0; Uhat = U."""
    d, g, M = P.mesh.dim, P.gamma, P.mach
    p = T / (g * M * M)
    u = np.zeros(d + 2)
    u[0] = 1.0
    u[-1] = p / (g - 1.0)
    P.U = np.broadcast_to(u[None, :, None], P.U.shape).copy()
    P.Ustar = P.U.copy()
    P.Q = np.zeros_like(P.Q)
    P.UH = np.broadcast_to(u[None, :, None], P.UH.shape).copy()
    return P


@pytest.mark.parametrize("dim,p", [(2, 2), (3, 1)])
def test_rest_state_in_wall_boxes(dim, p):
    for tag, T, Tw in ((3, 1.3, 1.3), (4, 0.7, 5.0)):
        P = synth.tiny(dim, p, periodic=False, visc_law=1, av=1e-3)
        P = with_tags(rest_state(P, T), {(r, s): tag for r in range(dim) for s in (0, 1)})
        P.twall = Tw
        pb = Problem(P)
        Rq, Ru, Rh = pb.global_residual(pb.Q, pb.U, pb.UH)
        sc = np.abs(pb.U).max()
        assert max(np.abs(Rq).max(), np.abs(Ru).max(), np.abs(Rh).max()) < 1e-13 * sc, tag


def test_uniform_stream_through_inflow_and_outflow():
    P = synth.tiny(2, 2, periodic=(False, True))
    P = with_tags(P, {(0, 0): 1, (0, 1): 2})
    ub = synth.freestream(2, P.gamma, P.mach)
    P.U = np.broadcast_to(ub[None, :, None], P.U.shape).copy()
    P.Ustar = P.U.copy()
    P.Q = np.zeros_like(P.Q)
    P.UH = np.broadcast_to(ub[None, :, None], P.UH.shape).copy()
    P.ubc = ub
    pb = Problem(P)
    Rq, Ru, Rh = pb.global_residual(pb.Q, pb.U, pb.UH)
    assert max(np.abs(Rq).max(), np.abs(Ru).max(), np.abs(Rh).max()) < 1e-13 * np.abs(ub).max()
    assert (P.mesh.bnd_tag == 2).any() and (P.mesh.bnd_tag == 1).any()


@pytest.mark.parametrize("tag", [3, 4])
def test_wall_box_conserves_at_convergence(tag):
    P = synth.tiny(2, 1, seed=5, periodic=False, visc_law=1, mach=0.4)
    P = with_tags(P, {(r, s): tag for r in range(2) for s in (0, 1)})
    P.twall = 1.1
    P.Ustar = P.U.copy()
    pb = Problem(P)
    Q, U, UH, hist = newton(pb, pb.Q, pb.U, pb.UH, tol=1e-11, maxit=12)
    assert hist[-1] <= 1e-11
    w = np.stack([pb.geom(e).M.sum(axis=1) for e in range(P.mesh.n_elem)])
    dI = np.einsum("ei,eai->a", w, U - P.Ustar)
    scale = np.abs(np.einsum("ei,eai->a", w, U - P.U)).max() + np.abs(U - P.U).max()
    assert abs(dI[0]) < 1e-9 * max(scale, 1e-300)
    if tag == 4:
        assert abs(dI[-1]) < 1e-9 * max(scale, 1e-300)
    assert np.abs(U - P.U).max() > 1e-6          # Newton moved the state


@pytest.mark.parametrize("tags", [{(0, 0): 1, (0, 1): 2}, {(1, 0): 3, (1, 1): 1}, {(1, 0): 4, (1, 1): 4}],
                         ids=["inflow-outflow", "isothermal-farfield", "adiabatic"])
def test_condensation_equals_global_solve_with_boundaries(tags):
    per = (True, False) if (1, 0) in tags else (False, True)
    P = synth.tiny(2, 2, periodic=per, visc_law=1, av=1e-3)
    P = with_tags(P, tags)
    P.twall = 0.9
    brute_force(P)
