"""The oracle's lifted gradient (eq. hdg-grad solved for Q) against closed forms.

For a polynomial state of total degree <= p and a trace equal to the exact
trace of that state, integration by parts turns the gradient equations into
(q - grad u, phi)_K = 0, so the lifted gradient is the exact gradient at the
nodes.  Checked on sheared (parallelepiped) meshes with Dirichlet sides, in
2-D and 3-D, p = 1..3; plus R_q(Q_lift) = 0 for a random state.
"""
import numpy as np
import pytest

import synth
from oracle.hdg import Problem


def poly_state(dim, p, seed):
    """m random polynomials of total degree <= p in x, with their gradients."""
    rng = np.random.default_rng(seed)
    m = dim + 2
    exps = [e for e in np.ndindex(*(p + 1,) * dim) if sum(e) <= p]
    coef = rng.normal(size=(m, len(exps)))

    def u(x):
        out = np.zeros(x.shape[:-1] + (m,))
        for c, e in enumerate(exps):
            mono = np.prod([x[..., k] ** e[k] for k in range(dim)], axis=0)
            out += coef[:, c] * mono[..., None]
        return out

    def grad(x):
        out = np.zeros(x.shape[:-1] + (dim, m))
        for c, e in enumerate(exps):
            for k in range(dim):
                if e[k] == 0:
                    continue
                ee = list(e)
                ee[k] -= 1
                mono = e[k] * np.prod([x[..., j] ** ee[j] for j in range(dim)], axis=0)
                out[..., k, :] += coef[:, c] * mono[..., None]
        return out

    return u, grad


def sheared_problem(dim, p, seed=0):
    P = synth.tiny(dim, p, periodic=False)
    mesh = P.mesh
    xyz = mesh.vert_xyz.copy()
    xyz[:, 0] += 0.3 * xyz[:, 1]
    if dim == 3:
        xyz[:, 2] += 0.2 * xyz[:, 0] - 0.1 * xyz[:, 1]
    mesh.vert_xyz = xyz
    return P


def exact_trace(pb, x, u_nodes):
    """Uhat[F][m][Nfp] from element nodal values (continuous across faces)."""
    r, cn = pb.ref, pb.conn
    UH = np.zeros((cn.n_faces, r.m, r.Nfp))
    for e in range(x.shape[0]):
        for f in range(r.nf):
            F = cn.e2f[e, f]
            UH[F][:, cn.perm[e, f]] = u_nodes[e][:, r.fnode[f]]
    return UH


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_lift_is_exact_gradient_of_polynomials(dim, p):
    P = sheared_problem(dim, p)
    pb = Problem(P)
    x = synth.node_xyz(P.mesh, p)                       # [E][Np][d]
    u, grad = poly_state(dim, p, seed=10 * dim + p)
    U = np.ascontiguousarray(u(x).transpose(0, 2, 1))   # [E][m][Np]
    UH = exact_trace(pb, x, U)
    Q = pb.lift_gradient(U, UH)
    G = grad(x).transpose(0, 2, 3, 1)                   # [E][d][m][Np]
    assert np.abs(Q - G).max() <= 1e-11 * np.abs(G).max()


def test_lift_zeroes_gradient_residual():
    P = synth.tiny(2, 3, periodic=(True, False))
    pb = Problem(P)
    Q = pb.lift_gradient(pb.U, pb.UH)
    Rq, _, _ = pb.global_residual(Q, pb.U, pb.UH)
    Rq0, _, _ = pb.global_residual(pb.Q, pb.U, pb.UH)
    assert np.abs(Rq).max() < 1e-13 * np.abs(Rq0).max()
