"""Pins of the state-dependent stabilization option tau(uhat) = |vhat.n| + chat + mu / h.

The wave-speed part is pinned against the spectral radius of the normal
convective flux Jacobian computed numerically (complex step + eigenvalues);
the residuals with tau(uhat) against finite differences of the Jacobians, the
brute-force condensation, and freestream preservation.
"""
import numpy as np
import pytest

import synth
from oracle import tet as ot
from oracle.hdg import Problem
from oracle.physics import Physics, convective_flux, stabilization, viscosity
from synth import tetmesh as tm


@pytest.mark.parametrize("law", [0, 1])
def test_wave_speed_part_is_the_spectral_radius(law):
    ph = Physics(1.4, 200.0, 0.72, 0.7, law, 1.4042, 0.40417)
    rng = np.random.default_rng(3)
    for _ in range(10):
        rho = 0.5 + rng.random()
        v = rng.standard_normal(3)
        p = 0.5 + rng.random()
        u = np.concatenate([[rho], rho * v, [p / 0.4 + 0.5 * rho * v @ v]])
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        A = np.zeros((5, 5))
        for b in range(5):
            uc = u.astype(complex)
            uc[b] += 1e-30j
            A[:, b] = (convective_flux(uc, ph) @ n).imag / 1e-30
        radius = np.abs(np.linalg.eigvals(A)).max()
        h = 0.3
        tau = stabilization(u, n, h, ph)
        assert abs(tau - viscosity(u, ph) / h - radius) < 1e-12 * radius


def test_hex_jacobian_with_state_dependent_tau_matches_fd():
    P = synth.tiny(2, 2, seed=7)
    P.tau_mode = 1
    pb = Problem(P)
    R, J = pb.element_jacobian(4)
    r = pb.ref
    Qe, Ue, UHe = pb.Q[4], pb.U[4], pb.local_trace(pb.UH, 4)
    x0 = np.concatenate([Qe.ravel(), Ue.ravel(), UHe.ravel()])
    nq, nu_ = Qe.size, Ue.size

    def res(x):
        a, b, c = pb.element_residual(4, x[:nq].reshape(Qe.shape), x[nq:nq + nu_].reshape(Ue.shape),
                                      x[nq + nu_:].reshape(UHe.shape))
        return np.concatenate([a.ravel(), b.ravel(), c.ravel()])

    for cidx in np.random.default_rng(1).choice(x0.size, 10, replace=False):
        h = 1e-6 * max(1.0, abs(x0[cidx]))
        xp, xm = x0.copy(), x0.copy()
        xp[cidx] += h
        xm[cidx] -= h
        fd = (res(xp) - res(xm)) / (2 * h)
        assert np.allclose(fd, J[:, cidx], atol=1e-6 * max(1.0, np.abs(J[:, cidx]).max()))
    assert r.m == 4


def test_tau_option_changes_the_blocks_but_keeps_freestream():
    P = synth.tiny(2, 1, seed=5)
    cond0 = Problem(P).condense(0)
    P.tau_mode = 1
    pb = Problem(P)
    cond1 = pb.condense(0)
    assert np.linalg.norm(cond1["S"] - cond0["S"]) > 1e-3 * np.linalg.norm(cond0["S"])
    ub = P.ubc
    U = np.broadcast_to(ub[None, :, None], P.U.shape).copy()
    UH = np.broadcast_to(ub[None, :, None], P.UH.shape).copy()
    pb.Ustar = U
    a, b, c = pb.global_residual(np.zeros_like(P.Q), U, UH)
    assert max(np.abs(a).max(), np.abs(b).max(), np.abs(c).max()) < 1e-12


def test_tet_condensation_with_state_dependent_tau_is_consistent():
    """Brute force on a curved mixed-degree tet mesh with tau(uhat)."""
    mesh = tm.kuhn_box((2, 1, 1), [np.linspace(0, 1, 3), np.linspace(0, .5, 2), np.linspace(0, .5, 2)],
                       (False, False, False), bump=tm.wall_bump(0.05), curved_layers=1, seed=3, pmax=2)
    prob = tm.config4_problem(mesh)
    prob.tau_mode = 1
    conn = ot.TetConnectivity(mesh)
    prob.U, prob.Q, prob.UH, prob.Ustar = tm.packed_state(mesh, tm.sinusoids(1.4, 0.5, 3, 1e-3), conn.nfp,
                                                          prob.ubc, 5)
    pb = ot.TetProblem(prob)
    e = 0
    R, J = pb.element_jacobian(e)
    Qe, Ue, UHe = pb.views(e)
    x0 = np.concatenate([Qe.ravel(), Ue.ravel()] + [h.ravel() for h in UHe])
    nq, nu_ = Qe.size, Ue.size
    sizes = [h.size for h in UHe]

    def res(x):
        uh, o = [], nq + nu_
        for f in range(4):
            uh.append(x[o:o + sizes[f]].reshape(UHe[f].shape))
            o += sizes[f]
        a, b, c = pb.element_residual(e, x[:nq].reshape(Qe.shape), x[nq:nq + nu_].reshape(Ue.shape), uh)
        return np.concatenate([a.ravel(), b.ravel()] + [h.ravel() for h in c])

    for cidx in range(nq + nu_, x0.size, 7):       # trace columns: where d tau / d uhat enters
        h = 1e-6 * max(1.0, abs(x0[cidx]))
        xp, xm = x0.copy(), x0.copy()
        xp[cidx] += h
        xm[cidx] -= h
        fd = (res(xp) - res(xm)) / (2 * h)
        assert np.allclose(fd, J[:, cidx], atol=1e-6 * max(1.0, np.abs(J[:, cidx]).max()))
