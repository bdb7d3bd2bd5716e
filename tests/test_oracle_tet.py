"""Pins of the tetrahedral oracle (mixed degree, quadratic geometry).

Each check compares the oracle with something it does not compute itself:
closed-form integrals of barycentric monomials, the Lagrange property,
orthonormality, exact differentiation of polynomials, the divergence theorem
on a curved mesh, freestream preservation, the conservation identity, the
brute-force uncondensed solve, finite differences, the geometric
consistency of the two sides of every face, and the consistency order on an
exact steady Navier-Stokes solution.
"""
import math

import numpy as np
import pytest

import synth
from oracle import tet as ot
from synth import tetmesh as tm


def bary_integral(ex, dim):
    """int over the reference simplex of prod lambda_i^{e_i} (Dirichlet integral)."""
    vol = 4.0 / 3.0 if dim == 3 else 2.0
    num = math.factorial(dim) * np.prod([math.factorial(e) for e in ex])
    return vol * num / math.factorial(sum(ex) + dim)


def tet_bary(x):
    return np.stack([-(1 + x[:, 0] + x[:, 1] + x[:, 2]) / 2, (1 + x[:, 0]) / 2, (1 + x[:, 1]) / 2,
                     (1 + x[:, 2]) / 2], axis=1)


def tri_bary(x):
    return np.stack([-(x[:, 0] + x[:, 1]) / 2, (1 + x[:, 0]) / 2, (1 + x[:, 1]) / 2], axis=1)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_tet_rule_exact_to_degree_2n_minus_1(n):
    x, w = ot.tet_rule(n)
    lam = tet_bary(x)
    D = 2 * n - 1
    for a in range(D + 1):
        for b in range(D + 1 - a):
            for c in range(D + 1 - a - b):
                d = D - a - b - c           # top degree only, plus a few lower ones below
                for ex in ((a, b, c, d), (a, b, c, 0)):
                    val = w @ np.prod(lam ** np.array(ex), axis=1)
                    assert abs(val - bary_integral(ex, 3)) < 1e-14 * max(1.0, bary_integral(ex, 3)) + 1e-15


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_tri_rule_exact_to_degree_2n_minus_1(n):
    x, w = ot.tri_rule(n)
    lam = tri_bary(x)
    D = 2 * n - 1
    for a in range(D + 1):
        for b in range(D + 1 - a):
            for ex in ((a, b, D - a - b), (a, b, 0)):
                val = w @ np.prod(lam ** np.array(ex), axis=1)
                assert abs(val - bary_integral(ex, 2)) < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_tet_basis_lagrange_orthonormal_and_exact_gradient(p):
    ref = ot.TetRef(p)
    assert ref.Np == len(tm.lattice(p)) == (p + 1) * (p + 2) * (p + 3) // 6
    assert np.allclose(ref.basis(ref.nodes), np.eye(ref.Np), atol=1e-12)
    assert np.allclose(ref.phi.sum(axis=1), 1.0, atol=1e-13)
    assert np.allclose(ref.dphi.sum(axis=2), 0.0, atol=1e-11)
    psi = ot.dubiner_tet(p, *ref.xq.T)
    assert np.allclose(psi.T @ (ref.wq[:, None] * psi), np.eye(ref.Np), atol=1e-12)
    # a degree-p polynomial is reproduced with its exact gradient
    rng = np.random.default_rng(p)
    c = rng.standard_normal((p + 1, p + 1, p + 1))

    def poly(x):
        return sum(c[i, j, k] * x[:, 0] ** i * x[:, 1] ** j * x[:, 2] ** k
                   for i in range(p + 1) for j in range(p + 1) for k in range(p + 1) if i + j + k <= p)

    def dpoly(x, r):
        out = np.zeros(len(x))
        for i in range(p + 1):
            for j in range(p + 1):
                for k in range(p + 1):
                    if i + j + k > p:
                        continue
                    e = [i, j, k]
                    if e[r] == 0:
                        continue
                    t = c[i, j, k] * e[r]
                    e[r] -= 1
                    out += t * x[:, 0] ** e[0] * x[:, 1] ** e[1] * x[:, 2] ** e[2]
        return out

    vals = poly(ref.nodes)
    assert np.allclose(ref.phi @ vals, poly(ref.xq), atol=1e-12)
    for r in range(3):
        assert np.allclose(ref.dphi[r] @ vals, dpoly(ref.xq, r), atol=1e-10)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_triangle_trace_basis(p):
    T = ot.TriRef(p)
    assert np.allclose(ot.dubiner_tri(p, *T.nodes.T) @ T.Vinv, np.eye(T.Nfp), atol=1e-12)
    assert np.allclose(T.mu.sum(axis=1), 1.0, atol=1e-13)
    M = T.mu.T @ (T.ws[:, None] * T.mu)
    assert abs(M.sum() - 2.0) < 1e-13                     # area of the reference triangle


def small_mesh(periodic=(False, False, False), n=(2, 1, 1), degrees=None, curved=True):
    coords = [np.linspace(0, 1, n[0] + 1), np.linspace(0, 0.5, n[1] + 1), np.linspace(0, 0.5, n[2] + 1)]
    return tm.kuhn_box(n, coords, periodic, bump=tm.wall_bump(0.05) if curved else None,
                       curved_layers=n[1] if curved else 0, degrees=degrees, seed=3)


def make_problem(mesh, seed=5, **kw):
    conn = ot.TetConnectivity(mesh)
    prob = tm.config4_problem(mesh, **kw)
    fun = tm.sinusoids(prob.gamma, prob.mach, 3, 1e-3)
    prob.U, prob.Q, prob.UH, prob.Ustar = tm.packed_state(mesh, fun, conn.nfp, prob.ubc, seed)
    return prob, ot.TetProblem(prob)


def test_kuhn_mesh_conforming_and_oriented():
    mesh = small_mesh(periodic=(True, False, True), n=(3, 1, 3))
    conn = ot.TetConnectivity(mesh)
    E = mesh.n_elem
    assert E == 6 * 9
    # every face has two elements except those on the y sides
    nb = int(np.sum(conn.f2e[:, 1, 0] < 0))
    assert nb == int(np.sum(mesh.bnd_tag > 0)) == 2 * 2 * 9
    assert 4 * E == 2 * conn.n_faces - nb
    for e in range(E):
        J = ot.p2_jacobian(mesh.geo[e], ot.TetRef(1).xq)
        assert np.all(np.linalg.det(J) > 0)
    # face degree is the larger element degree
    for F in range(conn.n_faces):
        ps = [mesh.elem_p[e] for (e, _) in conn.f2e[F] if e >= 0]
        assert conn.face_p[F] == max(ps)


def test_faces_match_geometrically_from_both_sides():
    """Canonical face points and area normals computed from the two elements of a
    face coincide (positions) and are opposite (normals), curved faces included."""
    mesh = small_mesh(n=(3, 2, 1), curved=True)
    conn = ot.TetConnectivity(mesh)
    T = ot.TriRef(3)
    for F in range(conn.n_faces):
        (e0, f0), (e1, f1) = conn.f2e[F]
        if e1 < 0:
            continue
        pts, nws = [], []
        for (e, f) in ((e0, f0), (e1, f1)):
            xi = ot.face_points(conn.L[e, f], T.xs)
            pts.append(ot.p2_map(mesh.geo[e], xi))
            Jf = ot.p2_jacobian(mesh.geo[e], xi)
            cof = np.linalg.det(Jf)[:, None, None] * np.transpose(np.linalg.inv(Jf), (0, 2, 1))
            nws.append(np.einsum("skr,r->sk", cof, ot.face_area_normal(f, conn.L[e, f])))
        assert np.allclose(pts[0], pts[1], atol=1e-14)
        assert np.allclose(nws[0], -nws[1], atol=1e-14)


def test_divergence_theorem_on_curved_mesh():
    """sum_K int_K 1 = (1/3) sum over boundary faces of int x . n (exact quadrature
    of the quadratic map: |J| has degree 3, x.n on a face degree 4)."""
    mesh = small_mesh(n=(2, 2, 1), degrees=2)
    prob, pb = make_problem(mesh)
    vol = sum(pb.geom(e).W.sum() for e in range(mesh.n_elem))
    flux = 0.0
    for e in range(mesh.n_elem):
        for f in range(4):
            if mesh.bnd_tag[e, f] == 0:
                continue
            G = pb.geom(e)
            T = pb.tri(pb.face_degrees(e)[f])
            x = ot.p2_map(mesh.geo[e], ot.face_points(pb.conn.L[e, f], T.xs))
            flux += np.sum(G.omega[f] * np.einsum("sk,sk->s", x, G.n[f])) / 3.0
    assert abs(vol - flux) < 1e-14 * vol
    assert abs(vol - 0.5 * 0.5 * 1.0) > 1e-6             # the bump changed the volume


@pytest.mark.parametrize("periodic", [(False, False, False), (True, False, True)])
def test_freestream_preserved_on_curved_mixed_mesh(periodic):
    n = (3, 1, 3) if periodic[0] else (2, 1, 1)
    mesh = small_mesh(periodic=periodic, n=n)
    prob, pb = make_problem(mesh)
    ub = prob.ubc
    c = pb.conn
    U = np.concatenate([np.repeat(ub, ot.n_tet(int(p))) for p in mesh.elem_p])
    UH = np.concatenate([np.repeat(ub, int(k)) for k in c.nfp])
    pb.Ustar = U
    a, b, h = pb.global_residual(np.zeros(3 * U.size), U, UH)
    assert np.abs(a).max() < 1e-13 and np.abs(b).max() < 1e-13 and np.abs(h).max() < 1e-13


def test_conservation_identity_periodic():
    mesh = small_mesh(periodic=(True, True, True), n=(3, 3, 3), curved=False)
    prob, pb = make_problem(mesh)
    c = pb.conn
    Rq, Ru, Rh = pb.global_residual(pb.Q, pb.U, pb.UH)
    lhs = np.zeros(5)
    for e in range(mesh.n_elem):
        Np, _ = pb.sizes(e)
        Ue = pb.U[c.uoff[e]:c.uoff[e + 1]].reshape(5, Np)
        Us = pb.Ustar[c.uoff[e]:c.uoff[e + 1]].reshape(5, Np)
        mass = (1.0 / pb.a_ii) * (Ue - Us) @ pb.geom(e).M.T
        lhs += (Ru[c.uoff[e]:c.uoff[e + 1]].reshape(5, Np) - mass).sum(axis=1)
    rhs = np.zeros(5)
    for F in range(c.n_faces):
        rhs += Rh[c.hoff[F]:c.hoff[F + 1]].reshape(5, -1).sum(axis=1)
    assert np.allclose(lhs, pb.dt * rhs, atol=1e-14, rtol=1e-12)


COUETTE_GAMMA, COUETTE_PR = 1.4, 0.72


def couette(x):
    return synth.couette_state(x - 0.5, COUETTE_GAMMA, COUETTE_PR)


def couette_gradient(x):
    """d u_a / d x_k of the Couette state, [..., 3, m], in closed form: only y varies,
    e = e0 - Pr y^2 / (2 gamma), rho = p0 / ((gamma - 1) e), rho v_x = rho y,
    rho E = p0 / (gamma - 1) + rho y^2 / 2 (p0 = 1, e0 = 2)."""
    g_, pr = COUETTE_GAMMA, COUETTE_PR
    y = x[..., 1] - 0.5
    e = 2.0 - pr * y * y / (2.0 * g_)
    rho = 1.0 / ((g_ - 1.0) * e)
    drho = rho / e * (pr * y / g_)
    out = np.zeros(x.shape[:-1] + (3, 5))
    out[..., 1, 0] = drho
    out[..., 1, 1] = rho + y * drho
    out[..., 1, 4] = 0.5 * y * y * drho + rho * y
    return out


def couette_residuals(n, p, curved):
    """Max-norm R_u, R_q (over h^3) and interior R_uhat (over h^2) with the exact
    Couette state interpolated at the element nodes and the trace nodes."""
    c = [np.linspace(0, 1, n + 1)] * 3
    mesh = tm.kuhn_box((n, n, n), c, (False, False, False), degrees=p,
                       bump=tm.wall_bump(0.05) if curved else None, curved_layers=n if curved else 0, seed=1)
    conn = ot.TetConnectivity(mesh)
    U, Q = [], []
    for e in range(mesh.n_elem):
        x = np.einsum("nc,ck->nk", tm.node_shape(p), mesh.geo[e])
        U.append(couette(x).T.ravel())
        Q.append(np.transpose(couette_gradient(x), (1, 2, 0)).ravel())
    U, Q = np.concatenate(U), np.concatenate(Q)
    UH = np.zeros(conn.hoff[-1])
    for F in range(conn.n_faces):
        e, f = conn.f2e[F, 0]
        xi = ot.face_points(conn.L[e, f], ot.TriRef(int(conn.face_p[F])).nodes)
        UH[conn.hoff[F]:conn.hoff[F + 1]] = couette(ot.p2_map(mesh.geo[e], xi)).T.ravel()
    prob = tm.TetProblem("couette", mesh, COUETTE_GAMMA, 20.0, COUETTE_PR, 0.5, 2.0, 1.0, 1.0, 0, 0.0, 0.0,
                         couette(np.zeros((1, 3)))[0])
    prob.U, prob.Q, prob.UH, prob.Ustar = U, Q, UH, U.copy()
    Rq, Ru, Rh = ot.TetProblem(prob).global_residual(Q, U, UH)
    h = 1.0 / n
    inner = np.concatenate([np.arange(conn.hoff[F], conn.hoff[F + 1]) for F in range(conn.n_faces)
                            if conn.f2e[F, 1, 0] >= 0])
    return np.abs(Ru).max() / h ** 3, np.abs(Rq).max() / h ** 3, np.abs(Rh[inner]).max() / h ** 2


def test_couette_gradient_closed_form():
    x = np.random.default_rng(0).uniform(0, 1, (20, 3))
    assert np.allclose(couette_gradient(x), synth.nodal_gradient(couette, x, 1e-5), rtol=0, atol=1e-8)


@pytest.mark.parametrize("p,curved,rate", [(2, False, 1.5), (3, False, 2.5), (3, True, 2.0)])
def test_couette_consistency_order(p, curved, rate):
    """Exact steady compressible NS solution (plane Couette flow with viscous
    heating) on affine and curved tetrahedra: the normalised element residuals
    fall at least at rate p - 1/2 (affine) or p - 1 (curved, pre-asymptotic: the
    wall bump keeps its amplitude as h halves) from 2^3 to 4^3 cells; a wrong
    flux, metric or lifting term leaves them O(1).  The interpolated trace is
    single valued and the element nodes restricted to a face are its trace
    nodes, so the two sides' face fluxes cancel: interior R_uhat vanishes to
    rounding on curved faces too."""
    r1 = couette_residuals(2, p, curved)
    r2 = couette_residuals(4, p, curved)
    for a, b in zip(r1[:2], r2[:2]):           # R_u, R_q
        assert b < a * 2.0 ** (-rate), (r1, r2)
    assert r1[2] < 1e-13 and r2[2] < 1e-13, (r1, r2)


def test_condensed_solve_equals_uncondensed_solve():
    """Brute force: the global Newton system J dW = -F solved densely equals
    the condensed trace solve plus element recovery."""
    mesh = small_mesh(n=(2, 1, 1))
    prob, pb = make_problem(mesh)
    c = pb.conn
    E = mesh.n_elem
    nint = [4 * 5 * pb.sizes(e)[0] for e in range(E)]
    ioff = np.concatenate([[0], np.cumsum(nint)])
    NT = int(c.hoff[-1])
    N = int(ioff[-1]) + NT
    J = np.zeros((N, N))
    F = np.zeros(N)
    vals, cache = pb.assemble()
    for e in range(E):
        R, Je = cache[e]["R"], cache[e]["J"]
        n = nint[e]
        gidx = list(range(ioff[e], ioff[e + 1]))
        for f, Fc in enumerate(c.e2f[e]):
            gidx += list(range(ioff[-1] + c.hoff[Fc], ioff[-1] + c.hoff[Fc + 1]))
        gidx = np.array(gidx)
        F[gidx[:n]] += R[:n]
        F[gidx[n:]] += R[n:]
        J[np.ix_(gidx, gidx)] += Je
    dW = np.linalg.solve(J, -F)
    # condensed
    S = np.zeros((NT, NT))
    for Fr in range(c.n_faces):
        for b in range(c.rowptr[Fr], c.rowptr[Fr + 1]):
            G = c.col[b]
            S[c.hoff[Fr]:c.hoff[Fr + 1], c.hoff[G]:c.hoff[G + 1]] = vals[b]
    g = pb.assemble_g(cache)
    dUH = np.linalg.solve(S, g)
    assert np.allclose(dUH, dW[ioff[-1]:], atol=1e-11 * np.abs(dW).max())
    for e in range(E):
        dQ, dU = pb.recover(e, cache[e], dUH)
        ref = dW[ioff[e]:ioff[e + 1]]
        got = np.concatenate([dQ.ravel(), dU.ravel()])
        assert np.allclose(got, ref, atol=1e-10 * np.abs(dW).max())


def test_jacobian_against_finite_differences():
    mesh = small_mesh(n=(2, 1, 1))
    prob, pb = make_problem(mesh)
    e = int(np.argmax(mesh.elem_p))
    R, J = pb.element_jacobian(e)
    Qe, Ue, UHe = pb.views(e)
    x0 = np.concatenate([Qe.ravel(), Ue.ravel()] + [h.ravel() for h in UHe])
    rng = np.random.default_rng(0)
    cols = rng.choice(x0.size, 12, replace=False)
    nq, nu_ = Qe.size, Ue.size
    sizes = [h.size for h in UHe]

    def res(x):
        q = x[:nq].reshape(Qe.shape)
        u = x[nq:nq + nu_].reshape(Ue.shape)
        uh, o = [], nq + nu_
        for f in range(4):
            uh.append(x[o:o + sizes[f]].reshape(UHe[f].shape))
            o += sizes[f]
        a, b, c = pb.element_residual(e, q, u, uh)
        return np.concatenate([a.ravel(), b.ravel()] + [h.ravel() for h in c])

    for cidx in cols:
        h = 1e-6 * max(1.0, abs(x0[cidx]))
        xp, xm = x0.copy(), x0.copy()
        xp[cidx] += h
        xm[cidx] -= h
        fd = (res(xp) - res(xm)) / (2 * h)
        assert np.allclose(fd, J[:, cidx], atol=1e-6 * max(1.0, np.abs(J[:, cidx]).max()))


def test_uniform_degree_affine_elements_share_reference_blocks():
    """Translated copies of one affine element with one state give identical S^K
    (a linear-algebra identity of the uniform case)."""
    mesh = small_mesh(periodic=(True, True, True), n=(3, 3, 3), degrees=2, curved=False)
    prob, pb = make_problem(mesh)
    c = pb.conn
    ub = prob.ubc
    pb.U = np.concatenate([np.repeat(ub, ot.n_tet(2)) for _ in range(mesh.n_elem)])
    pb.Ustar = pb.U.copy()
    pb.Q = np.zeros(3 * pb.U.size)
    pb.UH = np.concatenate([np.repeat(ub, int(k)) for k in c.nfp])
    # elements 0 and 6 * 13 are the same Kuhn tet in two cells: same shape and orientation
    e0, e1 = 0, 6 * 13
    s0, s1 = pb.condense(e0)["S"], pb.condense(e1)["S"]
    # same canonical frames up to the cell shift: compare in the elements' own face order
    assert np.allclose(s0, s1, atol=1e-12 * np.abs(s0).max())


def test_tet_newton_converges_quadratically():
    """The oracle's Newton on a curved mixed-degree mesh: quadratic decrease of ||F||."""
    mesh = small_mesh(n=(2, 1, 1))
    prob, pb = make_problem(mesh)
    prob.Ustar = prob.U + 1e-3 * np.cos(np.arange(prob.U.size))
    pb = ot.TetProblem(prob)
    _, _, _, hist = ot.newton(pb, pb.Q, pb.U, pb.UH, tol=1e-12, maxit=6)
    assert hist[-1] < 1e-11
    rates = [np.log(hist[k + 1]) / np.log(hist[k]) for k in range(1, len(hist) - 1) if hist[k] < 1e-2]
    assert rates and min(rates) > 1.6
