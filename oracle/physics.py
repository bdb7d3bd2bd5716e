"""Compressible Navier-Stokes fluxes (Sec. 2.1), complex-step safe.

Oracle (test infrastructure only).  Every function accepts complex arrays so
that Jacobians can be taken by complex-step differentiation; nothing here uses
``abs``, ``max`` or branches on values.

Array conventions: ``u[..., a]`` conserved state (m = d + 2 components);
``q[..., a, k] = d u_a / d x_k`` (eq. mixed-variable); fluxes ``F[..., a, k]``,
component a in direction k.

Nondimensionalization (a reading; the paper leaves it to each case): freestream
rho = 1, |v| = 1, p = 1 / (gamma M^2); effective viscosity mu~ / Re; temperature
T~ = gamma M^2 p / rho = gamma (gamma - 1) M^2 e, so T~ = 1 in the freestream.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Physics:
    gamma: float
    re: float
    pr: float
    mach: float
    visc_law: int = 0        # 0: mu~ = 1;  1: Sutherland mu~ = C1 T^1.5 / (T + S)
    suth_c1: float = 1.4042
    suth_s: float = 0.40417


def primitives(u, gamma):
    """rho, v_i, E and p from u (eq. thermo-closure / ideal-gas)."""
    d = u.shape[-1] - 2
    rho = u[..., 0]
    v = u[..., 1:d + 1] / rho[..., None]
    E = u[..., d + 1] / rho
    p = (gamma - 1.0) * (u[..., d + 1] - 0.5 * rho * np.sum(v * v, axis=-1))
    return rho, v, E, p


def convective_flux(u, ph: Physics):
    """f^c_j = [rho v_j, rho v_i v_j + delta_ij p, rho H v_j] (eq. convective-flux)."""
    d = u.shape[-1] - 2
    rho, v, E, p = primitives(u, ph.gamma)
    F = np.zeros(u.shape + (d,), dtype=np.result_type(u, 1.0))
    for k in range(d):
        F[..., 0, k] = rho * v[..., k]
        for i in range(d):
            F[..., 1 + i, k] = rho * v[..., i] * v[..., k] + (p if i == k else 0.0)
        F[..., d + 1, k] = (rho * E + p) * v[..., k]  # rho H v_k with H = E + p / rho
    return F


def viscosity(u, ph: Physics):
    """Effective mu = mu~(T~) / Re; Sutherland per eq. sutherland / tgv-sutherland."""
    rho, v, E, p = primitives(u, ph.gamma)
    if ph.visc_law == 0:
        return np.ones_like(rho) / ph.re
    T = ph.gamma * ph.mach ** 2 * p / rho
    return ph.suth_c1 * T ** 1.5 / (T + ph.suth_s) / ph.re


def viscous_flux(u, q, nu, ph: Physics):
    """f^v_j = [0, tau_ij, v_i tau_ij + f_j] plus nu_AV q (eqs. viscous-flux, av-total).

    tau_ij = mu (d_j v_i + d_i v_j - 2/3 d_k v_k delta_ij), beta = 0 (Stokes);
    f_j = kappa d_j T = (gamma mu / Pr) d_j e since e = c_v T, kappa = c_p mu / Pr.
    Gradients of primitives from q: d_j v_i = (q_{i,j} - v_i q_{0,j}) / rho,
    d_j E = (q_{E,j} - E q_{0,j}) / rho, d_j e = d_j E - v_i d_j v_i.
    """
    d = u.shape[-1] - 2
    rho, v, E, p = primitives(u, ph.gamma)
    mu = viscosity(u, ph)
    dv = np.zeros(u.shape[:-1] + (d, d), dtype=np.result_type(u, q, 1.0))  # dv[..., i, j] = d_j v_i
    for i in range(d):
        for j in range(d):
            dv[..., i, j] = (q[..., 1 + i, j] - v[..., i] * q[..., 0, j]) / rho
    dE = (q[..., d + 1, :] - E[..., None] * q[..., 0, :]) / rho[..., None]
    de = dE - np.einsum("...i,...ij->...j", v, dv)
    div = sum(dv[..., i, i] for i in range(d))
    F = np.zeros(u.shape + (d,), dtype=np.result_type(u, q, 1.0))
    for i in range(d):
        for j in range(d):
            tau_ij = mu * (dv[..., i, j] + dv[..., j, i] - (2.0 / 3.0) * (div if i == j else 0.0))
            F[..., 1 + i, j] = tau_ij
            F[..., d + 1, j] = F[..., d + 1, j] + v[..., i] * tau_ij
    for j in range(d):
        F[..., d + 1, j] = F[..., d + 1, j] + ph.gamma * mu / ph.pr * de[..., j]
    if nu is not None:
        F = F + nu[..., None, None] * q
    return F


def numerical_flux(u, uh, q, nu, n, tau, ph: Physics):
    """fhat = (F^c(uhat) - F^v(uhat, q)) . n + tau (u - uhat) (eq. num-flux-hdg).

    ``u`` is the element's interior trace, ``uh`` the single-valued trace,
    ``q`` the element's gradient trace, ``n[..., k]`` the outward unit normal and
    ``tau`` a constant scalar (the reading of the face stabilization), or an
    array of one value per point (``[..., s]``, the state-dependent variant).
    """
    F = convective_flux(uh, ph) - viscous_flux(uh, q, nu, ph)
    tau = np.asarray(tau)
    if tau.ndim:
        tau = tau[..., None]
    return np.einsum("...ak,...k->...a", F, n) + tau * (u - uh)


def stabilization(uh, n, h, ph: Physics):
    """State-dependent stabilization tau = |vhat . n| + chat + mu(That) / h (Sec. 2.2
    describes it as a wave speed plus a viscous part over a length; h is the
    element's length scale |K|^{1/d}).  |x| is written sqrt(x^2) so that the
    complex-step derivative is sign(x) (x != 0)."""
    rho, v, E, p = primitives(uh, ph.gamma)
    vn = np.einsum("...k,...k->...", v, n)
    c = np.sqrt(ph.gamma * p / rho)
    return np.sqrt(vn * vn) + c + viscosity(uh, ph) / h
