"""Pins of the oracle's residuals, Jacobians and condensation (no GPU).

Each test checks the oracle against something other than itself: freestream
preservation, a discrete conservation identity, consistency on an exact
Navier-Stokes solution, finite differences, and the uncondensed global
Newton solve by brute force on tiny meshes.
"""
import copy

import numpy as np
import pytest

import synth
from oracle.hdg import Problem
from oracle.refelem import RefElem


def freestream_problem(dim, p, skew=0.0, visc_law=0, av=0.0):
    P = synth.tiny(dim, p, visc_law=visc_law, av=av)
    mesh = P.mesh
    if skew:
        xyz = mesh.vert_xyz.copy()
        xyz[:, 0] += skew * xyz[:, 1]          # affine shear: parallelogram elements
        mesh.vert_xyz = xyz
    ub = synth.freestream(dim, P.gamma, P.mach)
    P.U[:] = ub[None, :, None]
    P.Ustar[:] = P.U
    P.Q[:] = 0.0
    P.UH[:] = ub[None, :, None]
    return P


@pytest.mark.parametrize("dim,p,skew", [(2, 1, 0.0), (2, 2, 0.3), (2, 3, 0.0), (3, 1, 0.2), (3, 2, 0.0)])
def test_freestream_preservation(dim, p, skew):
    """Uniform u, q = 0, uhat = u on an affine mesh gives R = 0 (divergence theorem)."""
    P = freestream_problem(dim, p, skew, visc_law=1, av=1e-3)
    pb = Problem(P)
    Rq, Ru, Rh = pb.global_residual(pb.Q, pb.U, pb.UH)
    scale = np.abs(pb.U).max()
    assert np.abs(Rq).max() < 1e-13 * scale
    assert np.abs(Ru).max() < 1e-13 * scale
    assert np.abs(Rh).max() < 1e-13 * scale


@pytest.mark.parametrize("dim,p", [(2, 2), (3, 1)])
def test_discrete_conservation(dim, p):
    """sum_i R_u[a,i] - mass term = dt * sum_{F,l} R_uhat[F,a,l] (periodic mesh)."""
    P = synth.tiny(dim, p, av=2e-3, visc_law=1)
    pb = Problem(P)
    Rq, Ru, Rh = pb.global_residual(pb.Q, pb.U, pb.UH)
    mass = np.zeros(pb.ref.m)
    for e in range(P.mesh.n_elem):
        mass += (1.0 / pb.a_ii) * ((pb.U[e] - pb.Ustar[e]) @ pb.geom(e).M.T).sum(1)
    lhs = Ru.sum(axis=(0, 2)) - mass
    rhs = pb.dt * Rh.sum(axis=(0, 2))
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12 * np.abs(rhs).max())


def couette_residuals(dim, p, n):
    gamma, pr = 1.4, 0.72
    nn = (n,) * dim
    per = (True, False, True)[:dim]
    mesh = synth.box_mesh(dim, (max(n, 3),) + nn[1:], (0,) * dim, (1.0,) * dim, per)
    fun = lambda x: synth.couette_state(x - 0.5, gamma, pr)
    x = synth.node_xyz(mesh, p)
    U = np.ascontiguousarray(fun(x).transpose(0, 2, 1))
    Q = np.ascontiguousarray(synth.nodal_gradient(fun, x, 1e-6).transpose(0, 2, 3, 1))
    pb_in = synth.Problem("couette", mesh, p, gamma, 20.0, pr, 0.5, 2.0, 1.0, 1.0, 0, 0, 0,
                          U, Q, None, U.copy(), None, fun(np.zeros((1, dim)))[0])
    # exact trace: evaluate at the oracle's own face node positions
    from oracle.mesh import Connectivity
    cn = Connectivity(mesh, p)
    ref = RefElem(dim, p)
    UH = np.zeros((cn.n_faces, dim + 2, ref.Nfp))
    for F in range(cn.n_faces):
        e, f = cn.f2e[F][0]
        inv = np.argsort(cn.perm[e, f])
        UH[F] = fun(x[e, ref.fnode[f][inv]]).T
    pb_in.UH = UH
    pb = Problem(pb_in)
    Rq, Ru, Rh = pb.global_residual(pb.Q, pb.U, pb.UH)
    h = 1.0 / n
    interior = [F for F in range(cn.n_faces) if cn.f2e[F][1][0] >= 0]
    return (np.abs(Ru).max() / h ** dim, np.abs(Rq).max() / h ** dim,
            np.abs(Rh[interior]).max() / h ** (dim - 1))


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 3), (3, 2)])
def test_couette_consistency(dim, p):
    """Exact steady NS solution: normalized residuals vanish as h -> 0 at rate >= p - 1/2 (pre-asymptotic).

    A wrong flux term (sign, factor, index) leaves an O(1) normalized R_u.
    """
    ns = (4, 8) if dim == 2 else (3, 6)
    r1 = couette_residuals(dim, p, ns[0])
    r2 = couette_residuals(dim, p, ns[1])
    for a, b in zip(r1[:2], r2[:2]):       # R_u, R_q
        assert b < a * 2.0 ** (-p + 0.5), (r1, r2)
    assert r2[0] < 5e-3
    # the exact trace is single valued and q continuous: interior R_uhat vanishes
    assert r1[2] < 1e-12 and r2[2] < 1e-12


@pytest.mark.parametrize("dim,p,law,av", [(2, 2, 0, 0.0), (3, 1, 1, 1e-3)])
def test_jacobian_matches_finite_differences(dim, p, law, av):
    P = synth.tiny(dim, p, visc_law=law, av=av)
    pb = Problem(P)
    e = 4
    R, J = pb.element_jacobian(e)
    Qe, Ue, UHe = pb.Q[e], pb.U[e], pb.local_trace(pb.UH, e)
    x0 = np.concatenate([Qe.ravel(), Ue.ravel(), UHe.ravel()])

    def res(x):
        q = x[:Qe.size].reshape(Qe.shape)
        u = x[Qe.size:Qe.size + Ue.size].reshape(Ue.shape)
        uh = x[Qe.size + Ue.size:].reshape(UHe.shape)
        a, b, c = pb.element_residual(e, q, u, uh)
        return np.concatenate([a.ravel(), b.ravel(), c.ravel()])

    assert np.allclose(res(x0), R)
    cols = np.random.default_rng(0).choice(len(x0), 40, replace=False)
    for c in cols:
        h = 1e-6 * max(1.0, abs(x0[c]))
        dx = np.zeros_like(x0)
        dx[c] = h
        fd = (res(x0 + dx) - res(x0 - dx)) / (2 * h)
        assert np.allclose(J[:, c], fd, rtol=1e-6, atol=1e-6 * np.abs(J).max())


def brute_force(P):
    """Dense global Newton solve vs condensed solve + recovery."""
    pb = Problem(P)
    Q, U, UH = pb.Q, pb.U, pb.UH
    x0 = np.concatenate([Q.ravel(), U.ravel(), UH.ravel()])
    nQ, nU = Q.size, U.size

    def unpack(x):
        return (x[..., :nQ].reshape(x.shape[:-1] + Q.shape),
                x[..., nQ:nQ + nU].reshape(x.shape[:-1] + U.shape),
                x[..., nQ + nU:].reshape(x.shape[:-1] + UH.shape))

    def Fvec(x):
        a, b, c = pb.global_residual(*unpack(x))
        lead = x.shape[:-1]
        return np.concatenate([a.reshape(lead + (-1,)), b.reshape(lead + (-1,)), c.reshape(lead + (-1,))], -1)

    F0 = Fvec(x0)
    N = len(x0)
    J = np.zeros((N, N))
    for c0 in range(0, N, 512):
        c1 = min(N, c0 + 512)
        X = np.broadcast_to(x0.astype(complex), (c1 - c0, N)).copy()
        X[np.arange(c1 - c0), np.arange(c0, c1)] += 1e-30j
        J[:, c0:c1] = Fvec(X).imag.T / 1e-30
    dW = np.linalg.solve(J, -F0)
    dQ_ref, dU_ref, dUH_ref = unpack(dW)

    vals, cache = pb.assemble()
    cn = pb.conn
    bs = pb.ref.m * pb.ref.Nfp
    S = np.zeros((cn.n_faces * bs, cn.n_faces * bs))
    for F in range(cn.n_faces):
        for b in range(cn.rowptr[F], cn.rowptr[F + 1]):
            G = cn.col[b]
            S[F * bs:(F + 1) * bs, G * bs:(G + 1) * bs] = vals[b]
    g = np.concatenate([v.ravel() for v in pb.assemble_g(cache, range(cn.n_faces)).values()])
    dUH = np.linalg.solve(S, g).reshape(UH.shape)
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    assert rel(dUH, dUH_ref) < 1e-11
    for e in range(P.mesh.n_elem):
        dQ, dU = pb.recover(e, cache[e], dUH)
        assert rel(dU, dU_ref[e]) < 1e-10 * np.abs(dU_ref).max() / np.abs(dU_ref[e]).max()
        assert np.abs(dQ - dQ_ref[e]).max() < 1e-10 * np.abs(dQ_ref).max()
    # the same Jacobian against finite differences of the global residual
    rng = np.random.default_rng(1)
    for c in rng.choice(N, 12, replace=False):
        h = 1e-6 * max(1.0, abs(x0[c]))
        dx = np.zeros(N)
        dx[c] = h
        fd = (Fvec(x0 + dx) - Fvec(x0 - dx)) / (2 * h)
        assert np.allclose(J[:, c], fd, rtol=1e-6, atol=1e-6 * np.abs(J).max())


@pytest.mark.parametrize("dim,p,law,av", [(2, 1, 0, 0.0), (2, 2, 1, 2e-3), (3, 1, 0, 1e-3)])
def test_condensation_equals_global_solve(dim, p, law, av):
    brute_force(synth.tiny(dim, p, visc_law=law, av=av))


def test_condensation_with_dirichlet_boundary():
    brute_force(synth.tiny(2, 2, periodic=(True, False)))


def test_uniform_state_identical_element_blocks():
    P = freestream_problem(2, 2)
    P.U[:] += 0.01   # still uniform; residual nonzero through the mass term
    pb = Problem(P)
    S0 = pb.condense(0)["S"]
    for e in (1, 5, 8):
        assert np.allclose(pb.condense(e)["S"], S0, rtol=1e-12, atol=1e-12 * np.abs(S0).max())


@pytest.mark.parametrize("mach", [0.1, 1.25])
def test_tgv_initial_kinetic_energy(mach):
    """E_k(0) = 1/8 for the TGV state generator (Sec. 5.3 prints approximately 0.125)."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    mesh = synth.box_mesh(3, (6, 6, 6), (0,) * 3, (2 * np.pi,) * 3, (True,) * 3)
    ref = RefElem(3, 6)
    X = mesh.vert_xyz[mesh.elem_vert]
    h = 2 * np.pi / 6
    tot = 0.0
    for e in range(mesh.n_elem):
        x = X[e, 0] + (ref.xq + 1.0) * 0.5 * h
        u = synth.tgv_state(x, 1.4, mach)
        ke = 0.5 * (u[:, 1] ** 2 + u[:, 2] ** 2 + u[:, 3] ** 2) / u[:, 0]
        tot += ke @ ref.wq * (h / 2) ** 3
    ek = tot / (2 * np.pi) ** 3
    assert abs(ek - 0.125) < 1e-9
    assert abs(ek - gold["tgv_kinetic_energy_t0"]["value"]) < 1e-9


@pytest.mark.parametrize("dim,p", [(2, 2), (3, 1)])
def test_trace_residual_vanishes_at_average_trace(dim, p):
    """Element-wise constant states, q = 0, uhat = average of the two sides:
    the convective parts F(uhat).n cancel across every face and the
    stabilization parts sum to tau (uL + uR - 2 uhat) = 0, so R_uhat = 0."""
    P = synth.tiny(dim, p, visc_law=1, av=1e-3)
    pb = Problem(P)
    rng = np.random.default_rng(3)
    ub = synth.freestream(dim, P.gamma, P.mach)
    U = np.zeros_like(pb.U)
    for e in range(P.mesh.n_elem):
        U[e] = (ub * (1.0 + 0.05 * rng.normal(size=ub.shape)))[:, None]
    UH = np.zeros_like(pb.UH)
    cn = pb.conn
    for F in range(cn.n_faces):
        (e0, _), (e1, _) = cn.f2e[F]
        UH[F] = 0.5 * (U[e0][:, :1] + U[e1][:, :1])
    Rq, Ru, Rh = pb.global_residual(np.zeros_like(pb.Q), U, UH)
    assert np.abs(Rh).max() < 1e-13 * np.abs(U).max()
