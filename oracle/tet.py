"""Tetrahedral HDG elements of per-element degree on quadratic geometry, in plain FP64.

Oracle (test infrastructure only).  The batched workload of the method's
evaluation (curved, anisotropic tetrahedral meshes with a mix of degrees,
Sec. 4) read as follows:

* element space: polynomials of total degree p_K on each tetrahedron (the
  spaces of Sec. 2.2); nodal Lagrange basis on the equispaced lattice of
  degree p_K, built from the orthonormal Dubiner basis through its
  Vandermonde matrix (values in collapsed coordinates, gradients by complex
  step);
* trace space of a face: total degree p_F = max(p_L, p_R) (the reading for
  mixed degrees; p_F = p_K on boundary faces), Lagrange on the equispaced
  lattice of the face triangle in the face's canonical frame: its vertices in
  ascending master vertex id g0 < g1 < g2, node (i, j) at barycentric weights
  ((p_F - i - j) / p_F, i / p_F, j / p_F) on (g0, g1, g2);
* quadrature: collapsed Gauss-Jacobi rules, p + 2 points per collapsed
  direction in the element (exact to degree 2p + 3) and p_F + 2 on each face;
  face points are placed in the canonical frame, so the two elements of a face
  integrate at the same physical points and each element's trace unknowns are
  in canonical order (no permutation);
* geometry: the isoparametric quadratic map of 10 nodes per element
  (vertices, then the midpoints of edges 01, 02, 03, 12, 13, 23), evaluated at
  every quadrature point: w |J|, J^{-1}, and face normals by Nanson's formula
  omega n = w cof(J) nu_ref with nu_ref the reference area normal of the face
  parametrisation;
* residuals, Jacobians (complex step), condensation, assembly, matvec and
  recovery as in ``oracle.hdg`` (Sec. 2.2-2.5), with per-element sizes.

Reference tetrahedron: vertices v0 = (-1,-1,-1), v1 = (1,-1,-1),
v2 = (-1,1,-1), v3 = (-1,-1,1); local face f is opposite vertex f.
Element nodes (i, j, k), i + j + k <= p, at xi = -1 + 2 (i, j, k) / p, k
slowest, i fastest.  Element unknowns ``[Q (d, m, Np) | U (m, Np)]``; element
trace unknowns ``(f, a, l)`` face by face, each face m x Nfp(p_F).
"""
from __future__ import annotations

import numpy as np
from scipy.special import roots_jacobi

from .mesh import master
from .physics import Physics, convective_flux, numerical_flux, stabilization, viscous_flux

H_CS = 1e-30

TET_VERTS = np.array([[-1.0, -1.0, -1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]])
TET_FACES = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))
TET_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
TET_OUTWARD = np.array([[1.0, 1.0, 1.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0], [0.0, 0.0, -1.0]])


def n_tet(p: int) -> int:
    return (p + 1) * (p + 2) * (p + 3) // 6


def n_tri(p: int) -> int:
    return (p + 1) * (p + 2) // 2


def tet_lattice(p: int):
    return [(i, j, k) for k in range(p + 1) for j in range(p + 1 - k) for i in range(p + 1 - j - k)]


def tri_lattice(p: int):
    return [(i, j) for j in range(p + 1) for i in range(p + 1 - j)]


def tet_nodes(p: int) -> np.ndarray:
    return np.array([[-1.0 + 2.0 * c / p for c in ijk] for ijk in tet_lattice(p)])


def tri_nodes(p: int) -> np.ndarray:
    return np.array([[-1.0 + 2.0 * c / p for c in ij] for ij in tri_lattice(p)])


# ----------------------------------------------------------------------------
# orthonormal Dubiner bases (collapsed coordinates)
# ----------------------------------------------------------------------------
def jacobi_orthonormal(n: int, alpha: int, x):
    """P_n^{(alpha,0)}(x), orthonormal for the weight (1 - x)^alpha on [-1, 1].

    Three-term recurrence of the Jacobi polynomials (beta = 0); complex-safe.
    """
    x = np.asarray(x)
    p0 = np.ones_like(x)
    if n == 0:
        pn = p0
    else:
        p1 = 0.5 * ((alpha + 2.0) * x + alpha)
        pm, pn = p0, p1
        for k in range(2, n + 1):
            a1 = 2.0 * k * (k + alpha) * (2.0 * k + alpha - 2.0)
            a2 = (2.0 * k + alpha - 1.0) * alpha * alpha
            a3 = (2.0 * k + alpha - 2.0) * (2.0 * k + alpha - 1.0) * (2.0 * k + alpha)
            a4 = 2.0 * (k + alpha - 1.0) * (k - 1.0) * (2.0 * k + alpha)
            pm, pn = pn, ((a2 + a3 * x) * pn - a4 * pm) / a1
    return pn / np.sqrt(2.0 ** (alpha + 1) / (2.0 * n + alpha + 1.0))


def _collapse_ratio(num, den):
    """num / den - 1 mapped to -1 where den = 0 (the collapsed vertex / edge)."""
    den = np.asarray(den)
    safe = np.where(np.abs(den) > 1e-14, den, 1.0)
    return np.where(np.abs(den) > 1e-14, num / safe - 1.0, -1.0)


def dubiner_tri(p: int, r, s):
    """psi[n, m] of the orthonormal triangle basis, m over ``tri_lattice(p)``."""
    r, s = np.asarray(r), np.asarray(s)
    a = _collapse_ratio(2.0 * (1.0 + r), 1.0 - s)
    b = s
    out = []
    for (i, j) in tri_lattice(p):
        out.append(2.0 ** (i + 0.5) * jacobi_orthonormal(i, 0, a) * ((1.0 - b) / 2.0) ** i
                   * jacobi_orthonormal(j, 2 * i + 1, b))
    return np.stack(out, axis=-1)


def dubiner_tet(p: int, x, y, z):
    """psi[n, m] of the orthonormal tetrahedron basis, m over ``tet_lattice(p)``."""
    x, y, z = np.asarray(x), np.asarray(y), np.asarray(z)
    a = _collapse_ratio(2.0 * (1.0 + x), -y - z)
    b = _collapse_ratio(2.0 * (1.0 + y), 1.0 - z)
    c = z
    out = []
    for (i, j, k) in tet_lattice(p):
        out.append(2.0 ** (2 * i + j + 1.5) * jacobi_orthonormal(i, 0, a) * ((1.0 - b) / 2.0) ** i
                   * jacobi_orthonormal(j, 2 * i + 1, b) * ((1.0 - c) / 2.0) ** (i + j)
                   * jacobi_orthonormal(k, 2 * i + 2 * j + 2, c))
    return np.stack(out, axis=-1)


# ----------------------------------------------------------------------------
# collapsed Gauss-Jacobi rules
# ----------------------------------------------------------------------------
def tet_rule(n: int):
    """Points [n^3, 3] and weights of the collapsed rule on the reference tet.

    xi = (1+a)(1-b)(1-c)/4 - 1, eta = (1+b)(1-c)/2 - 1, zeta = c; the collapse
    Jacobian ((1-b)/2)((1-c)/2)^2 is absorbed by Gauss-Jacobi weights with
    alpha = 1 (b) and alpha = 2 (c).  Order: c slowest, a fastest.
    """
    a, wa = roots_jacobi(n, 0, 0)
    b, wb = roots_jacobi(n, 1, 0)
    c, wc = roots_jacobi(n, 2, 0)
    pts, w = [], []
    for kc in range(n):
        for kb in range(n):
            for ka in range(n):
                pts.append([(1 + a[ka]) * (1 - b[kb]) * (1 - c[kc]) / 4 - 1, (1 + b[kb]) * (1 - c[kc]) / 2 - 1, c[kc]])
                w.append(wa[ka] * wb[kb] * wc[kc] / 8.0)
    return np.array(pts), np.array(w)


def tri_rule(n: int):
    """Points [n^2, 2] and weights of the collapsed rule on the reference triangle."""
    a, wa = roots_jacobi(n, 0, 0)
    b, wb = roots_jacobi(n, 1, 0)
    pts, w = [], []
    for kb in range(n):
        for ka in range(n):
            pts.append([(1 + a[ka]) * (1 - b[kb]) / 2 - 1, b[kb]])
            w.append(wa[ka] * wb[kb] / 2.0)
    return np.array(pts), np.array(w)


class TetRef:
    """Nodal Lagrange basis of degree p on the reference tetrahedron."""

    def __init__(self, p: int):
        self.p = p
        self.Np = n_tet(p)
        self.nodes = tet_nodes(p)
        V = dubiner_tet(p, *self.nodes.T)
        self.Vinv = np.linalg.inv(V)
        self.xq, self.wq = tet_rule(p + 2)
        self.Nq = len(self.wq)
        self.phi = self.basis(self.xq)
        self.dphi = self.grad(self.xq)

    def basis(self, x):
        x = np.asarray(x)
        return dubiner_tet(self.p, x[:, 0], x[:, 1], x[:, 2]) @ self.Vinv

    def grad(self, x):
        """dphi[r, n, j] = d phi_j / d xi_r at interior points (complex step)."""
        out = np.zeros((3, len(x), self.Np))
        for r in range(3):
            xc = np.asarray(x, complex).copy()
            xc[:, r] += 1j * H_CS
            out[r] = (dubiner_tet(self.p, xc[:, 0], xc[:, 1], xc[:, 2]) @ self.Vinv).imag / H_CS
        return out


class TriRef:
    """Trace basis of degree pF on the canonical face triangle, at its rule points."""

    def __init__(self, pF: int):
        self.p = pF
        self.Nfp = n_tri(pF)
        self.nodes = tri_nodes(pF)
        self.Vinv = np.linalg.inv(dubiner_tri(pF, *self.nodes.T))
        self.xs, self.ws = tri_rule(pF + 2)
        self.Nfq = len(self.ws)
        self.mu = dubiner_tri(pF, *self.xs.T) @ self.Vinv


def face_points(L, rs):
    """Reference-tet points of canonical face coordinates rs [n, 2] on the face
    whose canonical vertices are the local vertices L = (L0, L1, L2)."""
    m1 = (1.0 + rs[:, 0]) / 2.0
    m2 = (1.0 + rs[:, 1]) / 2.0
    m0 = 1.0 - m1 - m2
    V = TET_VERTS
    return m0[:, None] * V[L[0]] + m1[:, None] * V[L[1]] + m2[:, None] * V[L[2]]


def face_area_normal(f: int, L) -> np.ndarray:
    """d xi / d r x d xi / d s of the canonical parametrisation, oriented outward."""
    V = TET_VERTS
    nu = np.cross((V[L[1]] - V[L[0]]) / 2.0, (V[L[2]] - V[L[0]]) / 2.0)
    return nu if nu @ TET_OUTWARD[f] > 0 else -nu


# ----------------------------------------------------------------------------
# quadratic geometry
# ----------------------------------------------------------------------------
def p2_shape(xi):
    """Values N[n, 10] and reference derivatives dN[n, 10, 3] of the quadratic tet."""
    xi = np.asarray(xi)
    lam = np.stack([-(1.0 + xi[:, 0] + xi[:, 1] + xi[:, 2]) / 2.0, (1.0 + xi[:, 0]) / 2.0,
                    (1.0 + xi[:, 1]) / 2.0, (1.0 + xi[:, 2]) / 2.0], axis=1)
    dlam = np.array([[-0.5, -0.5, -0.5], [0.5, 0.0, 0.0], [0.0, 0.5, 0.0], [0.0, 0.0, 0.5]])
    N = np.zeros((len(xi), 10))
    dN = np.zeros((len(xi), 10, 3))
    for i in range(4):
        N[:, i] = lam[:, i] * (2.0 * lam[:, i] - 1.0)
        dN[:, i, :] = (4.0 * lam[:, i] - 1.0)[:, None] * dlam[i]
    for c, (a, b) in enumerate(TET_EDGES):
        N[:, 4 + c] = 4.0 * lam[:, a] * lam[:, b]
        dN[:, 4 + c, :] = 4.0 * (lam[:, a][:, None] * dlam[b] + lam[:, b][:, None] * dlam[a])
    return N, dN


def p2_jacobian(X10, xi):
    """J[n, k, r] = d x_k / d xi_r of the quadratic map with nodes X10 [10, 3]."""
    _, dN = p2_shape(xi)
    return np.einsum("ncr,ck->nkr", dN, X10)


def p2_map(X10, xi):
    N, _ = p2_shape(xi)
    return N @ X10


# ----------------------------------------------------------------------------
# connectivity
# ----------------------------------------------------------------------------
class TetConnectivity:
    """Faces, canonical frames, face degrees and the block pattern of a tet mesh.

    * faces numbered by first encounter scanning e = 0.., local f = 0..3;
    * ``f2e[F] = [(e, f), (e', f')]`` with (-1, -1) on boundary faces;
    * ``L[e, f]`` the local vertices of face f in ascending master id (the
      canonical frame of the face);
    * ``face_p[F] = max(p_e)`` over its elements; ``hoff`` trace offsets
      (m Nfp per face);
    * block row F: the faces of the elements touching F, ascending; each block
      sums its element contributions in ascending element id.
    """

    def __init__(self, mesh, m: int = 5):
        ev = np.asarray(mesh.elem_vert)
        E = ev.shape[0]
        pmap = None if mesh.periodic_map is None else np.asarray(mesh.periodic_map)
        self.elem_p = np.asarray(mesh.elem_p, dtype=np.int64)
        faces = {}
        f2e = []
        self.e2f = np.zeros((E, 4), dtype=np.int64)
        self.L = np.zeros((E, 4, 3), dtype=np.int64)
        for e in range(E):
            mv = [master(pmap, int(v)) if pmap is not None else int(v) for v in ev[e]]
            if len(set(mv)) != 4:
                raise ValueError("element %d has repeated master vertices" % e)
            for f in range(4):
                loc = TET_FACES[f]
                key = tuple(sorted(mv[c] for c in loc))
                self.L[e, f] = sorted(loc, key=lambda c: mv[c])
                if key not in faces:
                    faces[key] = len(f2e)
                    f2e.append([(e, f)])
                else:
                    F = faces[key]
                    if len(f2e[F]) != 1:
                        raise ValueError("face shared by more than two elements")
                    f2e[F].append((e, f))
                self.e2f[e, f] = faces[key]
        self.n_faces = len(f2e)
        self.f2e = np.full((self.n_faces, 2, 2), -1, dtype=np.int64)
        for F, lst in enumerate(f2e):
            for s, ef in enumerate(lst):
                self.f2e[F, s] = ef
        self.face_p = np.array([max(self.elem_p[e] for (e, _) in lst) for lst in f2e], dtype=np.int64)
        self.nfp = np.array([n_tri(int(q)) for q in self.face_p], dtype=np.int64)
        self.hoff = np.concatenate([[0], np.cumsum(m * self.nfp)])
        npe = np.array([n_tet(int(q)) for q in self.elem_p])
        self.uoff = np.concatenate([[0], np.cumsum(m * npe)])
        self.qoff = np.concatenate([[0], np.cumsum(3 * m * npe)])
        self.rowptr = [0]
        self.col = []
        for F in range(self.n_faces):
            cols = sorted({int(self.e2f[e, g]) for (e, _) in f2e[F] for g in range(4)})
            self.col.extend(cols)
            self.rowptr.append(len(self.col))
        self.rowptr = np.array(self.rowptr, dtype=np.int64)
        self.col = np.array(self.col, dtype=np.int64)
        self.contrib = []
        for F in range(self.n_faces):
            for b in range(self.rowptr[F], self.rowptr[F + 1]):
                G = self.col[b]
                lst = []
                for (e, fl) in sorted(f2e[F]):
                    for gl in range(4):
                        if self.e2f[e, gl] == G:
                            lst.append((e, fl, gl))
                self.contrib.append(lst)
        bs = m * self.nfp
        self.boff = np.concatenate([[0], np.cumsum([bs[F] * bs[self.col[b]] for F in range(self.n_faces)
                                                    for b in range(self.rowptr[F], self.rowptr[F + 1])])])

    def block_index(self, F: int, G: int) -> int:
        for b in range(self.rowptr[F], self.rowptr[F + 1]):
            if self.col[b] == G:
                return b
        raise KeyError((F, G))


# ----------------------------------------------------------------------------
# per-element geometry and tables
# ----------------------------------------------------------------------------
class TetGeometry:
    """Per-element tables: volume W, physical gradients, mass matrix; per face the
    element basis at the canonical face points, the trace basis, omega and n."""

    def __init__(self, ref: TetRef, tri: list, L, X10):
        J = p2_jacobian(X10, ref.xq)
        det = np.linalg.det(J)
        if np.any(det <= 0):
            raise ValueError("non-positive Jacobian")
        Jinv = np.linalg.inv(J)                                    # [g, r, k] = d xi_r / d x_k
        self.W = ref.wq * det
        self.dphi = np.einsum("rgi,grk->gik", ref.dphi, Jinv)       # [g, i, k]
        self.M = np.einsum("g,gi,gj->ij", self.W, ref.phi, ref.phi)
        self.phif, self.mu, self.omega, self.n = [], [], [], []
        for f in range(4):
            T = tri[f]
            xi = face_points(L[f], T.xs)
            Jf = p2_jacobian(X10, xi)
            nu = face_area_normal(f, L[f])
            cof = np.linalg.det(Jf)[:, None, None] * np.transpose(np.linalg.inv(Jf), (0, 2, 1))
            nw = T.ws[:, None] * np.einsum("skr,r->sk", cof, nu)
            om = np.linalg.norm(nw, axis=1)
            self.phif.append(ref.basis(xi))
            self.mu.append(T.mu)
            self.omega.append(om)
            self.n.append(nw / om[:, None])


class TetProblem:
    """One stage linearization problem on a tetrahedral mesh of mixed degree.

    ``prob`` provides mesh (vert_xyz, elem_vert, periodic_map, bnd_tag [E][4],
    elem_p [E], geo [E][10][3]), gamma, re, pr, mach, visc_law, suth_c1,
    suth_s, tau, dt, a_ii, ubc (tag-1 state), twall, and the packed state:
    U [sum m Np], Q [sum 3 m Np] (per element [d][m][Np]), UH [sum m Nfp],
    Ustar like U.
    """

    def __init__(self, prob):
        mesh = prob.mesh
        self.m = 5
        self.conn = TetConnectivity(mesh, self.m)
        self.ph = Physics(prob.gamma, prob.re, prob.pr, prob.mach, prob.visc_law, prob.suth_c1, prob.suth_s)
        self.tau, self.dt, self.a_ii = prob.tau, prob.dt, prob.a_ii
        self.tau_mode = int(getattr(prob, "tau_mode", 0))     # 0 constant tau, 1 state-dependent
        self.U = np.asarray(prob.U, float)
        self.Q = np.asarray(prob.Q, float)
        self.UH = np.asarray(prob.UH, float)
        self.Ustar = np.asarray(prob.Ustar, float)
        self.ubc = None if getattr(prob, "ubc", None) is None else np.asarray(prob.ubc, float)
        self.bnd = np.zeros((len(self.conn.elem_p), 4), np.int64) if mesh.bnd_tag is None else np.asarray(mesh.bnd_tag)
        tw = getattr(prob, "twall", 1.0)
        self.e_wall = tw / (prob.gamma * (prob.gamma - 1.0) * prob.mach ** 2)
        self.geo = np.asarray(mesh.geo, float)
        self._ref, self._tri, self._geom = {}, {}, {}

    # ------------------------------------------------------------- tables
    def ref(self, p):
        if p not in self._ref:
            self._ref[p] = TetRef(p)
        return self._ref[p]

    def tri(self, p):
        if p not in self._tri:
            self._tri[p] = TriRef(p)
        return self._tri[p]

    def face_degrees(self, e):
        return [int(self.conn.face_p[self.conn.e2f[e, f]]) for f in range(4)]

    def geom(self, e):
        if e not in self._geom:
            p = int(self.conn.elem_p[e])
            self._geom[e] = TetGeometry(self.ref(p), [self.tri(q) for q in self.face_degrees(e)],
                                        self.conn.L[e], self.geo[e])
        return self._geom[e]

    # ------------------------------------------------------------- sizes
    def sizes(self, e):
        p = int(self.conn.elem_p[e])
        Np = n_tet(p)
        nfp = [n_tri(q) for q in self.face_degrees(e)]
        return Np, nfp

    def views(self, e, Q=None, U=None, UH=None):
        Q = self.Q if Q is None else Q
        U = self.U if U is None else U
        UH = self.UH if UH is None else UH
        Np, nfp = self.sizes(e)
        c = self.conn
        Qe = Q[..., c.qoff[e]:c.qoff[e + 1]].reshape(Q.shape[:-1] + (3, self.m, Np))
        Ue = U[..., c.uoff[e]:c.uoff[e + 1]].reshape(U.shape[:-1] + (self.m, Np))
        UHe = [UH[..., c.hoff[F]:c.hoff[F + 1]].reshape(UH.shape[:-1] + (self.m, nfp[f]))
               for f, F in enumerate(c.e2f[e])]
        return Qe, Ue, UHe

    # ------------------------------------------------------------- residual
    def element_residual(self, e, Qe, Ue, UHe):
        """R_q [..., 3, m, Np], R_u [..., m, Np], R_uhat^K (list over faces of [..., m, Nfp])."""
        ph, G = self.ph, self.geom(e)
        ref = self.ref(int(self.conn.elem_p[e]))
        Us = self.Ustar[self.conn.uoff[e]:self.conn.uoff[e + 1]].reshape(self.m, ref.Np)
        u_g = np.swapaxes(Ue @ ref.phi.T, -1, -2)                              # [..., g, a]
        q_g = np.swapaxes(np.moveaxis(Qe @ ref.phi.T, -1, -3), -1, -2)         # [..., g, a, k]
        Fl = convective_flux(u_g, ph) - viscous_flux(u_g, q_g, None, ph)
        Ru = (1.0 / self.a_ii) * (Ue - Us) @ G.M.T
        Ru = Ru - self.dt * np.einsum("g,...gak,gik->...ai", G.W, Fl, G.dphi, optimize=True)
        Rq = np.einsum("g,...gak,gi->...kai", G.W, q_g, ref.phi, optimize=True)
        Rq = Rq + np.einsum("g,...ga,gik->...kai", G.W, u_g, G.dphi, optimize=True)
        Rh = []
        for f in range(4):
            ph_f = G.phif[f]
            u_s = np.swapaxes(Ue @ ph_f.T, -1, -2)
            q_s = np.swapaxes(np.moveaxis(Qe @ ph_f.T, -1, -3), -1, -2)
            uh_s = np.swapaxes(UHe[f] @ G.mu[f].T, -1, -2)
            tau = self.tau if self.tau_mode == 0 else stabilization(uh_s, G.n[f], G.W.sum() ** (1.0 / 3.0), ph)
            fhat = numerical_flux(u_s, uh_s, q_s, None, G.n[f], tau, ph)
            Ru = Ru + self.dt * np.einsum("s,...sa,sj->...aj", G.omega[f], fhat, ph_f, optimize=True)
            Rq = Rq - np.einsum("s,...sa,sk,sj->...kaj", G.omega[f], uh_s, G.n[f], ph_f, optimize=True)
            tag = int(self.bnd[e, f])
            if tag == 0:
                bh = fhat
            elif tag == 1:
                bh = uh_s - self.ubc
            elif tag == 2:
                bh = uh_s - u_s
            elif tag in (3, 4):
                bh = uh_s.copy()
                bh[..., 0] = fhat[..., 0]
                if tag == 3:
                    bh[..., 4] = uh_s[..., 4] - uh_s[..., 0] * self.e_wall
                else:
                    bh[..., 4] = fhat[..., 4]
            else:
                raise ValueError("boundary tag %d not in the oracle" % tag)
            Rh.append(np.einsum("s,...sa,sl->...al", G.omega[f], bh, G.mu[f], optimize=True))
        return Rq, Ru, Rh

    # ------------------------------------------------------------- Jacobian
    def element_jacobian(self, e, Q=None, U=None, UH=None, chunk=256):
        Qe, Ue, UHe = self.views(e, Q, U, UH)
        x0 = np.concatenate([Qe.ravel(), Ue.ravel()] + [h.ravel() for h in UHe])
        N, nq, nu_ = x0.size, Qe.size, Ue.size
        sizes = [h.size for h in UHe]
        Rq, Ru, Rh = self.element_residual(e, Qe, Ue, UHe)
        R = np.concatenate([Rq.ravel(), Ru.ravel()] + [h.ravel() for h in Rh])
        J = np.zeros((N, N))
        for c0 in range(0, N, chunk):
            c1 = min(N, c0 + chunk)
            X = np.broadcast_to(x0.astype(complex), (c1 - c0, N)).copy()
            X[np.arange(c1 - c0), np.arange(c0, c1)] += 1j * H_CS
            q = X[:, :nq].reshape((c1 - c0,) + Qe.shape)
            u = X[:, nq:nq + nu_].reshape((c1 - c0,) + Ue.shape)
            uh, o = [], nq + nu_
            for f in range(4):
                uh.append(X[:, o:o + sizes[f]].reshape((c1 - c0,) + UHe[f].shape))
                o += sizes[f]
            a, b, c = self.element_residual(e, q, u, uh)
            Rc = np.concatenate([a.reshape(c1 - c0, -1), b.reshape(c1 - c0, -1)]
                                + [h.reshape(c1 - c0, -1) for h in c], axis=1)
            J[:, c0:c1] = Rc.imag.T / H_CS
        return R, J

    def condense(self, e, Q=None, U=None, UH=None):
        """S^K, g^K, X = A^{-1} B, y = A^{-1} R for element e (dense FP64 LU)."""
        R, J = self.element_jacobian(e, Q, U, UH)
        Np, _ = self.sizes(e)
        n = 4 * self.m * Np
        A, B, C, D = J[:n, :n], J[:n, n:], J[n:, :n], J[n:, n:]
        sol = np.linalg.solve(A, np.column_stack([B, R[:n]]))
        X, y = sol[:, :-1], sol[:, -1]
        return {"S": D - C @ X, "g": -R[n:] + C @ y, "X": X, "y": y, "R": R, "J": J}

    def element_trace_offsets(self, e):
        _, nfp = self.sizes(e)
        return np.concatenate([[0], np.cumsum([self.m * k for k in nfp])])

    # ------------------------------------------------------------- assembly
    def assemble(self, blocks=None):
        """Block values {b: [bs_F, bs_G]} (row-major semantic) and g (packed)."""
        c = self.conn
        blocks = range(len(c.col)) if blocks is None else blocks
        need = sorted({e for b in blocks for (e, _, _) in c.contrib[b]})
        cache = {e: self.condense(e) for e in need}
        vals = {}
        for b in blocks:
            F = int(np.searchsorted(c.rowptr, b, side="right") - 1)
            G = int(c.col[b])
            Sb = np.zeros((c.hoff[F + 1] - c.hoff[F], c.hoff[G + 1] - c.hoff[G]))
            for (e, fl, gl) in c.contrib[b]:
                o = self.element_trace_offsets(e)
                Sb = Sb + cache[e]["S"][o[fl]:o[fl + 1], o[gl]:o[gl + 1]]
            vals[b] = Sb
        return vals, cache

    def assemble_g(self, cache):
        c = self.conn
        g = np.zeros(c.hoff[-1])
        for F in range(c.n_faces):
            for (e, f) in sorted(tuple(x) for x in c.f2e[F] if x[0] >= 0):
                o = self.element_trace_offsets(e)
                g[c.hoff[F]:c.hoff[F + 1]] += cache[e]["g"][o[f]:o[f + 1]]
        return g

    def matvec(self, vals, x):
        c = self.conn
        y = np.zeros(c.hoff[-1])
        for F in range(c.n_faces):
            for b in range(c.rowptr[F], c.rowptr[F + 1]):
                G = c.col[b]
                y[c.hoff[F]:c.hoff[F + 1]] += vals[b] @ x[c.hoff[G]:c.hoff[G + 1]]
        return y

    def recover(self, e, cond_e, dUH):
        """dW_K = -y - X dUhat_K (eq. local-elimination): dQ_K [3, m, Np], dU_K [m, Np]."""
        c = self.conn
        dUHe = np.concatenate([dUH[c.hoff[F]:c.hoff[F + 1]] for F in c.e2f[e]])
        dW = -cond_e["y"] - cond_e["X"] @ dUHe
        Np, _ = self.sizes(e)
        nq = 3 * self.m * Np
        return dW[:nq].reshape(3, self.m, Np), dW[nq:].reshape(self.m, Np)

    # ------------------------------------------------------------- global
    def global_residual(self, Q, U, UH):
        """Packed [R_q], [R_u], [R_uhat] over the mesh (eq. nonlinear-residual)."""
        c = self.conn
        Rq, Ru, Rh = np.zeros_like(Q), np.zeros_like(U), np.zeros_like(UH)
        for e in range(len(c.elem_p)):
            Qe, Ue, UHe = self.views(e, Q, U, UH)
            a, b, h = self.element_residual(e, Qe, Ue, UHe)
            Rq[c.qoff[e]:c.qoff[e + 1]] = a.ravel()
            Ru[c.uoff[e]:c.uoff[e + 1]] = b.ravel()
            for f, F in enumerate(c.e2f[e]):
                Rh[c.hoff[F]:c.hoff[F + 1]] += h[f].ravel()
        return Rq, Ru, Rh


# ----------------------------------------------------------------------------
# Newton and DIRK on the tetrahedral stage equations (Sec. 2.3, 2.5)
# ----------------------------------------------------------------------------
def newton(pb: TetProblem, Q, U, UH, tol=1e-11, maxit=8, fixed=None):
    """Newton on the stage equations of pb (its Ustar, a_ii, dt): the condensed
    trace system assembled and solved densely, interiors recovered, unit step.
    Stops at ||F|| <= tol, or after exactly `fixed` iterations when given.
    Returns (Q, U, UH, history of ||F|| before each iteration and at the end)."""
    c = pb.conn
    Q, U, UH = (np.array(x, dtype=float, copy=True) for x in (Q, U, UH))
    hist = []
    nit = maxit if fixed is None else fixed
    NT = int(c.hoff[-1])
    for k in range(nit + 1):
        a, b, h = pb.global_residual(Q, U, UH)
        hist.append(float(np.sqrt(a @ a + b @ b + h @ h)))
        if k == nit or (fixed is None and hist[-1] <= tol):
            break
        pb.Q, pb.U, pb.UH = Q, U, UH
        vals, cache = pb.assemble()
        S = np.zeros((NT, NT))
        for F in range(c.n_faces):
            for bb in range(c.rowptr[F], c.rowptr[F + 1]):
                G = c.col[bb]
                S[c.hoff[F]:c.hoff[F + 1], c.hoff[G]:c.hoff[G + 1]] = vals[bb]
        dUH = np.linalg.solve(S, pb.assemble_g(cache))
        dQ, dU = np.zeros_like(Q), np.zeros_like(U)
        for e in range(len(c.elem_p)):
            q, u = pb.recover(e, cache[e], dUH)
            dQ[c.qoff[e]:c.qoff[e + 1]] = q.ravel()
            dU[c.uoff[e]:c.uoff[e + 1]] = u.ravel()
        Q, U, UH = Q + dQ, U + dU, UH + dUH
    return Q, U, UH, hist


def dirk_step(prob, A, b, tol=1e-11, maxit=8, fixed=None):
    """One DIRK step of the tetrahedral HDG system from (prob.Q, prob.U, prob.UH),
    each stage solved by Newton from the previous stage (oracle.dirk.dirk_step)."""
    from .dirk import dirk_step as generic_step
    pb = TetProblem(prob)
    Un = np.array(prob.U, dtype=float, copy=True)
    state = {"Q": np.array(prob.Q, float), "U": Un.copy(), "UH": np.array(prob.UH, float)}
    hists = []

    def solve_stage(i, Us, a_ii):
        pb.Ustar = Us
        pb.a_ii = a_ii
        Q, U, UH, h = newton(pb, state["Q"], state["U"], state["UH"], tol, maxit, fixed)
        state.update(Q=Q, U=U, UH=UH)
        hists.append(h)
        return U

    Unew, _ = generic_step(solve_stage, Un, A, b)
    return state["Q"], Unew, state["UH"], hists
