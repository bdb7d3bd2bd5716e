"""HDG stage residuals, Jacobians and static condensation, in plain FP64.

Oracle (test infrastructure only).  Follows Sec. 2.2-2.5:

* residuals of eq. hdg-weak with the DIRK mass term of eq. fully-discrete-local,
  written per element K (test functions r = e_k phi_i, w = e_a phi_i, mu_l):

    R_q[k,a,i] = (q_{a,k}, phi_i)_K + (u_a, d_k phi_i)_K - <uhat_a, phi_i n_k>_dK
    R_u[a,i]   = (1/a_ii) (M (U - U*))_{a,i}
                 + dt [ -(F^c - F^v)_{a,k}, d_k phi_i)_K + <fhat_a, phi_i>_dK ]
    R_uhat^K[f,a,l] = <fhat_a, mu_l>_F          (interior / periodic faces)
                    = <bhat_a, mu_l>_F            (boundary faces, readings of Sec. 2.2):
      tag 1 far-field / supersonic inflow  bhat = uhat - u_b
      tag 2 supersonic outflow             bhat = uhat - u
      tag 3 isothermal no-slip wall        bhat = [fhat_rho; uhat_rhov; uhat_rhoE - uhat_rho c_v T_w]
      tag 4 adiabatic no-slip wall         bhat = [fhat_rho; uhat_rhov; fhat_rhoE]

  with fhat = (F^c(uhat) - F^v(uhat, q)) . n + tau (u - uhat) (eq. num-flux-hdg)
  and a constant scalar tau (a reading of "face-based stabilization").
  U* = U^n - a_ii sum_{j<i} d_ij (U^{n,j} - U^n) is the known stage data
  (an exact rearrangement of eq. fully-discrete-local using d_ii = 1 / a_ii);
* Jacobians A = d(R_q, R_u)/d(Q, U), B = d(R_q, R_u)/d Uhat_K,
  C = d R_uhat^K / d(Q, U), D = d R_uhat^K / d Uhat_K, taken by complex-step
  differentiation of the residual (Squire & Trapp 1998), exact to rounding;
* condensation of eqs. newton-local-block, local-elimination, schur-trace read
  as A [dQ; dU] = -R - B dUhat_K, C [dQ; dU] + D dUhat_K = -R_uhat^K:
  X = A^{-1} B, y = A^{-1} R (dense LU with partial pivoting),
  S^K = D - C X, g^K = -R_uhat^K + C y, dW_K = -y - X dUhat_K.

Element unknown ordering: ``[Q (d, m, Np) | U (m, Np)]``; element trace dofs
``(f, a, l)`` with l in the element's local face frame.
"""
from __future__ import annotations

import numpy as np

from .mesh import Connectivity
from .physics import Physics, convective_flux, numerical_flux, stabilization, viscous_flux
from .refelem import RefElem

H_CS = 1e-30  # complex-step size


class Geometry:
    """Per-element geometric factors of the multilinear map (any quad / hex).

    ``x(xi) = sum_c N_c(xi) X_c`` with ``N_c = prod_r (1 +- xi_r) / 2``.
    Volume: ``W[g] = w_g |J_g|``, physical basis gradients ``dphi[g, i, k]``.
    Faces (Nanson): ``w_s |J| J^{-T} n_ref = omega_s n``.
    """

    def __init__(self, ref: RefElem, X: np.ndarray):
        d = ref.d
        self.X = X

        def jac(xi):  # jac[k, r] = d x_k / d xi_r
            J = np.zeros((d, d))
            for c in range(2 ** d):
                for r in range(d):
                    dN = 1.0
                    for s in range(d):
                        b = (c >> s) & 1
                        if s == r:
                            dN *= (0.5 if b else -0.5)
                        else:
                            dN *= 0.5 * (1.0 + xi[s]) if b else 0.5 * (1.0 - xi[s])
                    J[:, r] += dN * X[c]
            return J

        self.W = np.zeros(ref.Nq)
        self.dphi = np.zeros((ref.Nq, ref.Np, d))
        for g in range(ref.Nq):
            J = jac(ref.xq[g])
            Jinv = np.linalg.inv(J)  # Jinv[r, k] = d xi_r / d x_k
            self.W[g] = ref.wq[g] * np.linalg.det(J)
            self.dphi[g] = np.einsum("ri,rk->ik", ref.dphi[:, g, :], Jinv, optimize=True)
        self.omega = np.zeros((ref.nf, ref.Nfq))
        self.n = np.zeros((ref.nf, ref.Nfq, d))
        for f in range(ref.nf):
            for s in range(ref.Nfq):
                J = jac(ref.xf[f, s])
                Jinv = np.linalg.inv(J)
                nw = ref.wf[s] * np.linalg.det(J) * (Jinv.T @ ref.nref[f])
                self.omega[f, s] = np.linalg.norm(nw)
                self.n[f, s] = nw / self.omega[f, s]
        self.M = np.einsum("g,gi,gj->ij", self.W, ref.phi, ref.phi, optimize=True)


class Problem:
    """One stage linearization problem on a mesh: tables, geometry, data."""

    def __init__(self, prob):
        mesh = prob.mesh
        self.d = mesh.dim
        self.p = prob.p
        self.ref = RefElem(self.d, self.p)
        self.conn = Connectivity(mesh, self.p)
        self.ph = Physics(prob.gamma, prob.re, prob.pr, prob.mach, prob.visc_law, prob.suth_c1, prob.suth_s)
        self.tau = prob.tau
        self.tau_mode = int(getattr(prob, "tau_mode", 0))     # 0 constant tau, 1 state-dependent
        self.dt = prob.dt
        self.a_ii = prob.a_ii
        self.U = np.asarray(prob.U, float)
        self.Q = np.asarray(prob.Q, float)
        self.UH = np.asarray(prob.UH, float)
        self.Ustar = np.asarray(prob.Ustar, float)
        self.nu = None if prob.nu is None else np.asarray(prob.nu, float)
        self.ubc = None if prob.ubc is None else np.asarray(prob.ubc, float)
        self.bnd = np.asarray(mesh.bnd_tag)
        # wall internal energy c_v T_w = T~_w / (gamma (gamma - 1) M^2) (T~ = gamma M^2 p / rho)
        tw = getattr(prob, "twall", 1.0)
        self.e_wall = tw / (prob.gamma * (prob.gamma - 1.0) * prob.mach ** 2)
        self.X = mesh.vert_xyz[mesh.elem_vert]
        self._geom = {}
        r = self.ref
        self.nq_dofs = self.d * r.m * r.Np
        self.nu_dofs = r.m * r.Np
        self.n_int = self.nq_dofs + self.nu_dofs
        self.t = r.nf * r.m * r.Nfp

    def boundary_state(self, e: int, f: int):
        """u_b at the face quadrature points of a tag-1 face: a constant state
        [m], or nodal data [F][m][Nfp] in the face's canonical node order."""
        if self.ubc.ndim == 1:
            return self.ubc
        F = self.conn.e2f[e, f]
        return (self.ubc[F][:, self.conn.perm[e, f]] @ self.ref.mu.T).T

    def geom(self, e: int) -> Geometry:
        if e not in self._geom:
            self._geom[e] = Geometry(self.ref, self.X[e])
        return self._geom[e]

    # ------------------------------------------------------------------ traces
    def local_trace(self, UH: np.ndarray, e: int) -> np.ndarray:
        """Uhat_K [nf, m, Nfp] in the element's local face frames."""
        r = self.ref
        out = np.zeros((r.nf, r.m, r.Nfp), dtype=UH.dtype)
        for f in range(r.nf):
            F = self.conn.e2f[e, f]
            out[f] = UH[F][:, self.conn.perm[e, f]]
        return out

    # --------------------------------------------------------------- residual
    def element_residual(self, e: int, Qe, Ue, UHe):
        """R_q [..., d, m, Np], R_u [..., m, Np], R_uhat^K [..., nf, m, Nfp]."""
        r, ph, G = self.ref, self.ph, self.geom(e)
        nu_nodes = None if self.nu is None else self.nu[e]
        # volume (eqs. hdg-grad and hdg-cons)
        u_g = np.swapaxes(Ue @ r.phi.T, -1, -2)                      # [..., g, a]
        q_g = np.moveaxis(Qe @ r.phi.T, -1, -3)                      # [..., g, k, a]
        q_g = np.swapaxes(q_g, -1, -2)                               # [..., g, a, k]
        nu_g = None if nu_nodes is None else r.phi @ nu_nodes
        F = convective_flux(u_g, ph) - viscous_flux(u_g, q_g, nu_g, ph)
        Ru = (1.0 / self.a_ii) * (Ue - self.Ustar[e]) @ G.M.T
        Ru = Ru - self.dt * np.einsum("g,...gak,gik->...ai", G.W, F, G.dphi, optimize=True)
        Rq = np.einsum("g,...gak,gi->...kai", G.W, q_g, r.phi, optimize=True)
        Rq = Rq + np.einsum("g,...ga,gik->...kai", G.W, u_g, G.dphi, optimize=True)
        Rh = np.zeros(Ue.shape[:-2] + (r.nf, r.m, r.Nfp), dtype=np.result_type(Qe, Ue, UHe, 1.0))
        for f in range(r.nf):
            u_s = np.swapaxes(Ue @ r.phif[f].T, -1, -2)              # [..., s, a]
            q_s = np.swapaxes(np.moveaxis(Qe @ r.phif[f].T, -1, -3), -1, -2)
            uh_s = np.swapaxes(UHe[..., f, :, :] @ r.mu.T, -1, -2)   # [..., s, a]
            nu_s = None if nu_nodes is None else r.phif[f] @ nu_nodes
            tau = self.tau if self.tau_mode == 0 else stabilization(uh_s, G.n[f], G.W.sum() ** (1.0 / self.d), ph)
            fhat = numerical_flux(u_s, uh_s, q_s, nu_s, G.n[f], tau, ph)
            Ru = Ru + self.dt * np.einsum("s,...sa,sj->...aj", G.omega[f], fhat, r.phif[f], optimize=True)
            Rq = Rq - np.einsum("s,...sa,sk,sj->...kaj", G.omega[f], uh_s, G.n[f], r.phif[f], optimize=True)
            tag = int(self.bnd[e, f])
            if tag == 0:
                bh = fhat
            elif tag == 1:                       # far-field / supersonic inflow: all variables prescribed
                bh = uh_s - self.boundary_state(e, f)
            elif tag == 2:                       # supersonic outflow: interior state extrapolated
                bh = uh_s - u_s
            elif tag in (3, 4):                  # no-slip wall: mass flux, uhat_v = 0, thermal condition
                d = self.d
                bh = uh_s.copy()
                bh[..., 0] = fhat[..., 0]
                if tag == 3:                     # isothermal: rho e = rho c_v T_w at vhat = 0
                    bh[..., d + 1] = uh_s[..., d + 1] - uh_s[..., 0] * self.e_wall
                else:                            # adiabatic: zero normal energy flux
                    bh[..., d + 1] = fhat[..., d + 1]
            else:
                raise ValueError("boundary tag %d not in the oracle" % tag)
            Rh[..., f, :, :] = np.einsum("s,...sa,sl->...al", G.omega[f], bh, r.mu, optimize=True)
        return Rq, Ru, Rh

    # --------------------------------------------------------------- Jacobian
    def element_jacobian(self, e: int, Q=None, U=None, UH=None, chunk: int = 256):
        """Residual vector and Jacobian of [R_q; R_u; R_uhat^K] w.r.t. [Q_K; U_K; Uhat_K]."""
        Q = self.Q if Q is None else Q
        U = self.U if U is None else U
        UH = self.UH if UH is None else UH
        r = self.ref
        Qe, Ue, UHe = Q[e], U[e], self.local_trace(UH, e)
        x0 = np.concatenate([Qe.ravel(), Ue.ravel(), UHe.ravel()])
        N = x0.size
        nq, nu_ = Qe.size, Ue.size
        Rq, Ru, Rh = self.element_residual(e, Qe, Ue, UHe)
        R = np.concatenate([Rq.ravel(), Ru.ravel(), Rh.ravel()])
        J = np.zeros((N, N))
        for c0 in range(0, N, chunk):
            c1 = min(N, c0 + chunk)
            X = np.broadcast_to(x0.astype(complex), (c1 - c0, N)).copy()
            X[np.arange(c1 - c0), np.arange(c0, c1)] += 1j * H_CS
            q = X[:, :nq].reshape((c1 - c0,) + Qe.shape)
            u = X[:, nq:nq + nu_].reshape((c1 - c0,) + Ue.shape)
            uh = X[:, nq + nu_:].reshape((c1 - c0,) + UHe.shape)
            a, b, c = self.element_residual(e, q, u, uh)
            Rc = np.concatenate([a.reshape(c1 - c0, -1), b.reshape(c1 - c0, -1), c.reshape(c1 - c0, -1)], axis=1)
            J[:, c0:c1] = Rc.imag.T / H_CS
        return R, J

    # ----------------------------------------------------------- condensation
    def condense(self, e: int, Q=None, U=None, UH=None):
        """S^K, g^K, X = A^{-1}B, y = A^{-1}R for element e (dense FP64 LU)."""
        R, J = self.element_jacobian(e, Q, U, UH)
        n = self.n_int
        A, B, C, D = J[:n, :n], J[:n, n:], J[n:, :n], J[n:, n:]
        sol = np.linalg.solve(A, np.column_stack([B, R[:n]]))
        X, y = sol[:, :-1], sol[:, -1]
        return {"S": D - C @ X, "g": -R[n:] + C @ y, "X": X, "y": y, "A": A, "B": B, "C": C, "D": D, "R": R}

    # --------------------------------------------------------------- assembly
    def assemble(self, elems=None, blocks=None):
        """Assembled BSR values (semantic row-major ``[nnzb][b][b]``) and g.

        Only the blocks listed in ``blocks`` (default: all) are formed, from the
        elements that touch them; each block sums its contributions in
        ascending element order.
        """
        r, cn = self.ref, self.conn
        bsz = r.m * r.Nfp
        blocks = range(len(cn.col)) if blocks is None else blocks
        need = sorted({e for b in blocks for (e, _, _) in cn.contrib[b]})
        if elems is not None:
            need = sorted(set(need) | set(elems))
        cache = {e: self.condense(e) for e in need}
        vals = {}
        for b in blocks:
            Sb = np.zeros((bsz, bsz))
            for (e, fl, gl) in cn.contrib[b]:
                SK = cache[e]["S"].reshape(r.nf, r.m, r.Nfp, r.nf, r.m, r.Nfp)
                blk = SK[fl, :, :, gl, :, :]                         # [a, l, b, l']
                pr, pc = cn.perm[e, fl], cn.perm[e, gl]
                tmp = np.zeros((r.m, r.Nfp, r.m, r.Nfp))
                tmp[:, pr[:, None], :, pc[None, :]] = np.transpose(blk, (1, 3, 0, 2))
                Sb = Sb + tmp.reshape(bsz, bsz)
            vals[b] = Sb
        return vals, cache

    def assemble_g(self, cache, faces):
        r, cn = self.ref, self.conn
        out = {}
        for F in faces:
            gF = np.zeros((r.m, r.Nfp))
            for (e, f) in cn.f2e[F]:
                if e < 0:
                    continue
                gK = cache[int(e)]["g"].reshape(r.nf, r.m, r.Nfp)
                tmp = np.zeros((r.m, r.Nfp))
                tmp[:, cn.perm[e, f]] = gK[f]
                gF = gF + tmp
            out[F] = gF
        return out

    # ------------------------------------------------------------ trace ops
    def matvec(self, vals, x):
        """y_F = sum_G S_FG x_G over the block pattern (Sec. 3.2 trace operator)."""
        cn = self.conn
        F = cn.n_faces
        xv = x.reshape(F, -1)
        y = np.zeros_like(xv)
        for Fi in range(F):
            for b in range(cn.rowptr[Fi], cn.rowptr[Fi + 1]):
                y[Fi] = y[Fi] + vals[b] @ xv[cn.col[b]]
        return y.reshape(x.shape)

    def recover(self, e: int, cond_e, dUH):
        """dW_K = -y - X dUhat_K (eq. local-elimination): returns dQ_K, dU_K."""
        dUHe = self.local_trace(dUH, e).ravel()
        dW = -cond_e["y"] - cond_e["X"] @ dUHe
        r = self.ref
        dQ = dW[:self.nq_dofs].reshape(self.d, r.m, r.Np)
        dU = dW[self.nq_dofs:].reshape(r.m, r.Np)
        return dQ, dU

    def lift_gradient(self, U, UH):
        """Q for which R_q = 0 on every element (eq. hdg-grad).

        R_q is affine in Q with dR_q/dQ = I (x) M_K, so
        Q_K = -M_K^{-1} R_q(0, U_K, Uhat_K), one solve per (k, a).
        """
        r = self.ref
        E = U.shape[0]
        Q = np.zeros((E, self.d, r.m, r.Np))
        zero = np.zeros((self.d, r.m, r.Np))
        for e in range(E):
            Rq0 = self.element_residual(e, zero, U[e], self.local_trace(UH, e))[0]
            rhs = -Rq0.reshape(self.d * r.m, r.Np).T
            Q[e] = np.linalg.solve(self.geom(e).M, rhs).T.reshape(self.d, r.m, r.Np)
        return Q

    # -------------------------------------------------------- global system
    def global_residual(self, Q, U, UH):
        """[R_q; R_u; R_uhat] over the whole mesh (eq. nonlinear-residual)."""
        r, cn = self.ref, self.conn
        E = Q.shape[-4]
        lead = Q.shape[:-4]
        dt = np.result_type(Q, U, UH, 1.0)
        Rq = np.zeros(Q.shape, dtype=dt)
        Ru = np.zeros(U.shape, dtype=dt)
        Rh = np.zeros(UH.shape, dtype=dt)
        for e in range(E):
            UHe = np.zeros(lead + (r.nf, r.m, r.Nfp), dtype=UH.dtype)
            for f in range(r.nf):
                UHe[..., f, :, :] = UH[..., cn.e2f[e, f], :, :][..., cn.perm[e, f]]
            a, b, c = self.element_residual(e, Q[..., e, :, :, :], U[..., e, :, :], UHe)
            Rq[..., e, :, :, :] = a
            Ru[..., e, :, :] = b
            for f in range(r.nf):
                F = int(cn.e2f[e, f])
                for lam in range(r.Nfp):
                    kap = int(cn.perm[e, f, lam])
                    Rh[..., F, :, kap] = Rh[..., F, :, kap] + c[..., f, :, lam]
        return Rq, Ru, Rh

    def residual_norm(self, Q=None, U=None, UH=None) -> float:
        Q = self.Q if Q is None else Q
        U = self.U if U is None else U
        UH = self.UH if UH is None else UH
        a, b, c = self.global_residual(Q, U, UH)
        return float(np.sqrt(np.sum(a * a) + np.sum(b * b) + np.sum(c * c)))
