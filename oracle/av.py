"""Artificial-viscosity sensor, its smoothing, and the TGV diagnostics, in FP64.

Oracle (test infrastructure only).  Follows Sec. 2.2, eq. av-coeffs, and
Sec. 5.1, eqs. tgv-kinetic-energy and tgv-total-dissipation.

Sensor (readings where the paper leaves the form open):
* at every solution node, from the nodal U and the nodal gradient Q:
  div = d_j v_j and omega = |curl v| with d_j v_i = (q_{i,j} - v_i q_{0,j}) / rho,
  c* = sqrt(gamma p / rho);
* L is the clamp to [0, upper]; the sensor responds to compression, so the
  divergence enters as L(-div); omega is already >= 0 and unbounded;
  the sensor value is clamped to [0, s_max];
      s = sqrt(h_m / k) * L(-div) / c* * L(-div)^2 / (L(-div)^2 + omega^2 + eps)
      nu_raw(node) = c_av * min(max(s, 0), s_max)
* the raw elemental value is the maximum over the element's nodes.
Smoothing S_h: average the elemental field to the (master) vertices, take the
element mean of its vertex values, average to the vertices again (two
vertex-averaging passes), then interpolate the vertex field multilinearly
(P1 / Q1) to the element's solution nodes.

Diagnostics, with the volume quadrature of the HDG discretisation:
  E_k = 1 / (2 |Omega|) int rho v.v,   eps_S = 1 / (Re |Omega|) int mu~ omega.omega,
  eps_D = 4 / (3 Re |Omega|) int mu~ (div v)^2,
with mu~ the nondimensional viscosity law (1 or Sutherland) and u, q the
interpolants of U, Q at the quadrature points.
"""
from __future__ import annotations

import numpy as np

from .hdg import Problem


def velocity_gradient(u, q):
    """u [..., m], q [..., d, m] (q[..., j, a] = d_j u_a) -> rho, v [..., d], G [..., i, j] = d_j v_i."""
    d = u.shape[-1] - 2
    rho = u[..., 0]
    v = u[..., 1:d + 1] / rho[..., None]
    G = np.zeros(u.shape[:-1] + (d, d))
    for i in range(d):
        for j in range(d):
            G[..., i, j] = (q[..., j, 1 + i] - v[..., i] * q[..., j, 0]) / rho
    return rho, v, G


def vorticity(G):
    d = G.shape[-1]
    if d == 2:
        return (G[..., 1, 0] - G[..., 0, 1])[..., None]
    return np.stack([G[..., 2, 1] - G[..., 1, 2], G[..., 0, 2] - G[..., 2, 0], G[..., 1, 0] - G[..., 0, 1]], -1)


def nodal_sensor(U, Q, gamma, c_av, h_m, k, s_max, eps=1e-12):
    """nu_raw at every node: [E][Np]."""
    u = np.moveaxis(U, -2, -1)                      # [E][Np][m]
    q = np.moveaxis(Q, -1, 1)                       # [E][Np][d][m]
    d = u.shape[-1] - 2
    rho, v, G = velocity_gradient(u, q)
    div = np.trace(G, axis1=-2, axis2=-1)
    om = np.linalg.norm(vorticity(G), axis=-1)
    p = (gamma - 1.0) * (u[..., d + 1] - 0.5 * rho * np.sum(v * v, axis=-1))
    c = np.sqrt(gamma * p / rho)
    Lc = np.maximum(-div, 0.0)
    s = np.sqrt(h_m / k) * Lc / c * Lc ** 2 / (Lc ** 2 + om ** 2 + eps)
    return c_av * np.clip(s, 0.0, s_max)


def element_masters(mesh):
    pm = np.asarray(mesh.periodic_map)
    ev = np.asarray(mesh.elem_vert)
    m = ev.copy()
    for _ in range(4):                              # periodic maps point to masters directly; be safe
        m = pm[m]
    return m


def smooth(mesh, nu_e, passes=2):
    """Vertex field after `passes` vertex-averaging passes of the elemental field."""
    ev = element_masters(mesh)
    nvert = mesh.n_vert
    cur = np.asarray(nu_e, float)
    for it in range(passes):
        acc = np.zeros(nvert)
        cnt = np.zeros(nvert)
        for e in range(ev.shape[0]):
            for v in ev[e]:
                acc[v] += cur[e]
                cnt[v] += 1
        nv = np.where(cnt > 0, acc / np.maximum(cnt, 1), 0.0)
        if it < passes - 1:
            cur = nv[ev].mean(axis=1)
    return nv


def interpolate_q1(mesh, p, nv, nodes1):
    """Multilinear interpolation of the vertex field to the nodes: [E][Np]."""
    ev = element_masters(mesh)
    d = mesh.dim
    n1 = p + 1
    t = 0.5 * (np.asarray(nodes1) + 1.0)
    out = np.zeros((ev.shape[0], n1 ** d))
    for i in range(n1 ** d):
        ii = [(i // n1 ** r) % n1 for r in range(d)]
        for c in range(2 ** d):
            w = 1.0
            for r in range(d):
                w *= t[ii[r]] if (c >> r) & 1 else 1.0 - t[ii[r]]
            out[:, i] += w * nv[ev[:, c]]
    return out


def av_field(P, U, Q, c_av, h_m, s_max, nodes1, passes=2):
    raw = nodal_sensor(U, Q, P.gamma, c_av, h_m, P.p, s_max).max(axis=1)
    return interpolate_q1(P.mesh, P.p, smooth(P.mesh, raw, passes), nodes1)


def tgv_diagnostics(P, U, Q):
    """(E_k, eps_S, eps_D, |Omega|) from the nodal state."""
    pb = Problem(P)
    r = pb.ref
    tot = np.zeros(4)
    for e in range(U.shape[0]):
        G_ = pb.geom(e)
        u = (U[e] @ r.phi.T).T                      # [Nq][m]
        q = np.einsum("kaj,gj->gka", Q[e], r.phi)   # [Nq][d][m]
        rho, v, G = velocity_gradient(u, q)
        mu = pb.ph.re * _viscosity(u, pb.ph)         # mu~ (viscosity() includes 1/Re)
        om = vorticity(G)
        div = np.trace(G, axis1=-2, axis2=-1)
        tot += np.array([G_.W @ (rho * np.sum(v * v, -1)), G_.W @ (mu * np.sum(om * om, -1)),
                         G_.W @ (mu * div ** 2), G_.W.sum()])
    vol = tot[3]
    re = P.re
    return tot[0] / (2 * vol), tot[1] / (re * vol), 4 * tot[2] / (3 * re * vol), vol


def _viscosity(u, ph):
    from .physics import viscosity
    return viscosity(u, ph)
