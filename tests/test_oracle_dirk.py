"""The oracle's DIRK driver against closed forms.

* Alexander's SDIRK3 tableau: every order condition up to order 3, the
  textbook value of its diagonal, stiff accuracy and L-stability.
* The generic step on the Dahlquist equation y' = lambda y, whose stage
  solves are exact, must reproduce the stability function
  R(z) = 1 + z b^T (I - z A)^{-1} 1 of the tableau, for a stiffly accurate
  tableau and for one that is not (the second exercises the weights e_j).
* On the HDG system: a uniform state is a fixed point, and a periodic mesh
  conserves the integral of every conserved variable over the step.
"""
import numpy as np
import pytest

import synth
from oracle.dirk import alexander_sdirk3, dirk_coefficients, dirk_step, hdg_dirk_step
from oracle.hdg import Problem


def stability_function(A, b, z):
    s = len(b)
    return 1.0 + z * b @ np.linalg.solve(np.eye(s) - z * A, np.ones(s))


def test_sdirk3_tableau():
    A, b, c = alexander_sdirk3()
    g = A[0, 0]
    # the diagonal of Alexander's method (Hairer & Wanner, Table IV.6.5)
    assert abs(g - 0.43586652150845899942) < 1e-15
    assert np.allclose(np.diag(A), g, rtol=0, atol=0)
    assert np.all(np.triu(A, 1) == 0)
    assert np.allclose(A.sum(axis=1), c, atol=1e-15)
    assert np.array_equal(A[-1], b)                       # stiffly accurate
    assert abs(b.sum() - 1) < 1e-15
    assert abs(b @ c - 1 / 2) < 1e-15
    assert abs(b @ c ** 2 - 1 / 3) < 1e-15
    assert abs(b @ A @ c - 1 / 6) < 1e-15                 # not imposed by the construction
    # L-stability: R(inf) = 1 - b^T A^{-1} 1 = 0 and |R(iy)| <= 1
    assert abs(1 - b @ np.linalg.solve(A, np.ones(3))) < 1e-14
    for y in np.logspace(-3, 4, 50):
        assert abs(stability_function(A, b, 1j * y)) <= 1 + 1e-14
    # third order and no more: b^T c^3 != 1/4
    assert abs(b @ c ** 3 - 1 / 4) > 1e-3


def two_stage_sdirk3():
    """Crouzeix's two-stage order-3 SDIRK, b = (1/2, 1/2): not stiffly accurate."""
    g = (3 + np.sqrt(3)) / 6
    A = np.array([[g, 0.0], [1 - 2 * g, g]])
    return A, np.array([0.5, 0.5])


@pytest.mark.parametrize("tab", ["alexander", "crouzeix"])
def test_dahlquist_reproduces_stability_function(tab):
    A, b = (alexander_sdirk3()[:2] if tab == "alexander" else two_stage_sdirk3())
    dt = 0.1
    for z in (-0.3, -2.0, -40.0, 0.5 + 1.5j, -1e-2 + 3j):
        lam = z / dt
        y0 = np.array([1.3 + 0.2j])
        # stage equations (1/a_ii)(U - U*) - dt lam U = 0, solved exactly
        out, stages = dirk_step(lambda i, Us, a: Us / (1.0 - a * dt * lam), y0, A, b)
        ref = stability_function(np.asarray(A, complex), np.asarray(b, complex), z) * y0
        assert np.allclose(out, ref, rtol=1e-13, atol=0)
        # each stage is Y_i = y0 + z sum_j a_ij Y_j
        Y = np.array([s_[0] for s_ in stages])
        assert np.allclose(Y, y0[0] + z * (A @ Y), rtol=1e-13, atol=0)


def test_dahlquist_third_order():
    A, b, _ = alexander_sdirk3()
    errs = []
    for dt in (0.04, 0.02, 0.01):
        lam = -1.7
        out, _ = dirk_step(lambda i, Us, a: Us / (1.0 - a * dt * lam), np.array([1.0]), A, b)
        errs.append(abs(out[0] - np.exp(lam * dt)))
    # local error O(dt^4)
    assert 14 < errs[0] / errs[1] < 18 and 14 < errs[1] / errs[2] < 18


def _mass_weights(pb):
    """Integral of each nodal basis function, per element: row sums of M_K."""
    return np.stack([pb.geom(e).M.sum(axis=1) for e in range(pb.U.shape[0])])


def test_hdg_dirk_uniform_state_is_fixed_point():
    P = synth.tiny(2, 1)
    ub = synth.freestream(2, P.gamma, P.mach)
    P.U = np.broadcast_to(ub[None, :, None], P.U.shape).copy()
    P.Q = np.zeros_like(P.Q)
    P.UH = np.broadcast_to(ub[None, :, None], P.UH.shape).copy()
    A, b, _ = alexander_sdirk3()
    Q, U, UH, hists = hdg_dirk_step(P, A, b, tol=1e-12)
    assert np.abs(U - P.U).max() < 1e-13 and np.abs(Q).max() < 1e-12 and np.abs(UH - P.UH).max() < 1e-13
    assert all(len(h) == 1 for h in hists)                # no Newton iteration needed


@pytest.mark.parametrize("tab", ["alexander", "crouzeix"])
def test_hdg_dirk_conserves_integrals_on_periodic_mesh(tab):
    A, b = (alexander_sdirk3()[:2] if tab == "alexander" else two_stage_sdirk3())
    P = synth.tiny(2, 1, seed=3)
    P.Ustar = P.U.copy()
    pb = Problem(P)
    w = _mass_weights(pb)
    before = np.einsum("ei,eai->a", w, P.U)
    Q, U, UH, hists = hdg_dirk_step(P, A, b, tol=1e-12)
    after = np.einsum("ei,eai->a", w, U)
    assert all(h[-1] <= 1e-12 for h in hists)
    assert np.abs(after - before).max() < 1e-11 * np.abs(before).max()
    # the step did something: the state moved by far more than the tolerance
    assert np.abs(U - P.U).max() > 1e-4
