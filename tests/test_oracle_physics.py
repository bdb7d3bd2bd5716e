"""Pins of the oracle's flux functions (Sec. 2.1) by invariants and closed forms."""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle.physics import Physics, convective_flux, primitives, viscosity, viscous_flux

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def rand_state(rng, d, n=6):
    rho = 0.8 + 0.4 * rng.random(n)
    v = rng.normal(size=(n, d))
    p = 0.5 + rng.random(n)
    u = synth.conserved(rho, [v[:, k] for k in range(d)], p, 1.4)
    q = rng.normal(size=(n, d + 2, d))
    return u, q


def rotation(rng):
    a = rng.normal(size=(3, 3))
    qm, _ = np.linalg.qr(a)
    return qm * np.sign(np.linalg.det(qm))


def rotate_state(R, u, q):
    d = R.shape[0]
    u2 = u.copy()
    u2[:, 1:d + 1] = u[:, 1:d + 1] @ R.T
    q2 = np.einsum("jk,nak->naj", R, q)             # rotate the derivative index
    q2[:, 1:d + 1, :] = np.einsum("il,nlj->nij", R, q2[:, 1:d + 1, :])
    return u2, q2


def rotate_flux(R, F):
    d = R.shape[0]
    G = np.einsum("jk,nak->naj", R, F)
    G[:, 1:d + 1, :] = np.einsum("il,nlj->nij", R, G[:, 1:d + 1, :])
    return G


@pytest.mark.parametrize("law", [0, 1])
def test_rotational_invariance(law):
    rng = np.random.default_rng(1)
    ph = Physics(1.4, 100.0, 0.72, 0.5, law)
    u, q = rand_state(rng, 3)
    R = rotation(rng)
    u2, q2 = rotate_state(R, u, q)
    assert np.allclose(convective_flux(u2, ph), rotate_flux(R, convective_flux(u, ph)), atol=1e-12)
    nu = rng.random(u.shape[0])
    assert np.allclose(viscous_flux(u2, q2, nu, ph), rotate_flux(R, viscous_flux(u, q, nu, ph)), atol=1e-12)


def test_stress_traceless_symmetric_and_zero_for_uniform():
    rng = np.random.default_rng(2)
    ph = Physics(1.4, 10.0, 0.72, 0.5)
    u, q = rand_state(rng, 3)
    F = viscous_flux(u, q, None, ph)
    tau = F[:, 1:4, :]
    assert np.allclose(np.einsum("nii->n", tau), 0.0, atol=1e-13)
    assert np.allclose(tau, np.swapaxes(tau, 1, 2), atol=1e-13)
    assert np.allclose(F[:, 0, :], 0.0)
    assert np.allclose(viscous_flux(u, 0 * q, None, ph), 0.0)


def test_heat_flux_closed_form():
    """Uniform velocity and a gradient of internal energy only: f_j = gamma mu / Pr de/dx_j."""
    ph = Physics(1.4, 7.0, 0.7, 0.5)
    rho, v, e = 1.3, np.array([0.4, -0.2, 0.1]), 2.0
    u = np.array([rho, *(rho * v), rho * (e + 0.5 * v @ v)])
    de = np.array([0.3, -0.7, 0.2])
    q = np.zeros((5, 3))
    q[4] = rho * de                       # d(rho E)/dx = rho de/dx when rho, v constant
    F = viscous_flux(u[None], q[None], None, ph)[0]
    assert np.allclose(F[4], 1.4 / 7.0 / 0.7 * de, atol=1e-14)
    assert np.allclose(F[1:4], 0.0, atol=1e-14)


def test_couette_pointwise_balance():
    """Plane Couette with heating: tau_12 = mu and the y energy flux vanishes."""
    gamma, pr = 1.4, 0.72
    ph = Physics(gamma, 50.0, pr, 0.5)
    y = np.linspace(-0.5, 0.5, 7)
    x = np.stack([0 * y, y, 0 * y], axis=1)
    fun = lambda x: synth.couette_state(x, gamma, pr)
    u = fun(x)
    q = np.swapaxes(synth.nodal_gradient(fun, x, 1e-6), -1, -2)
    F = viscous_flux(u, q, None, ph)
    mu = 1.0 / 50.0
    assert np.allclose(F[:, 1, 1], mu, atol=1e-8)        # tau_12 = mu dv1/dy
    assert np.allclose(F[:, 4, 1], 0.0, atol=1e-8)


def test_complex_step_matches_finite_differences():
    rng = np.random.default_rng(3)
    ph = Physics(1.4, 30.0, 0.72, 1.2, 1)
    u, q = rand_state(rng, 3, n=1)
    h = 1e-30
    f = lambda uu: convective_flux(uu, ph) - viscous_flux(uu, q.astype(complex), None, ph)
    for b in range(5):
        du = np.zeros(5)
        du[b] = 1.0
        cs = f(u + 1j * h * du).imag / h
        eps = 1e-6 * max(1.0, abs(u[0, b]))
        fd = (f(u + eps * du).real - f(u - eps * du).real) / (2 * eps)
        assert np.allclose(cs, fd, rtol=1e-6, atol=1e-6)


def test_sutherland_tgv_unit_temperature():
    """eq. tgv-sutherland at T = 1 gives mu~ = 1.4042 / 1.40417 (freestream T~ = 1)."""
    g = GOLD["tgv_sutherland"]
    ph = Physics(1.4, 1.0, 0.71, 1.25, 1, g["c1"], g["s"])
    u = synth.freestream(3, 1.4, 1.25)[None]
    assert abs(viscosity(u, ph)[0] - g["c1"] / (1.0 + g["s"])) < 1e-14


def test_table1_freestream_energy():
    """Table 1: rho = 1, p = 0.01446 gives E = p / (gamma - 1) + 1/2 = 0.53614 (to print precision)."""
    g = GOLD["mach7_freestream"]
    u = synth.conserved(np.array(g["rho"]), [np.array(1.0), np.array(0.0), np.array(0.0)], g["p"], 1.4)
    rho, v, E, p = primitives(u[None], 1.4)
    assert abs(E[0] - g["E"]) < 2e-5
    assert abs(p[0] - g["p"]) < 1e-15


@pytest.mark.parametrize("dim", [2, 3])
def test_convective_jacobian_eigenvalues(dim):
    """Textbook: d(F^c . n)/du has eigenvalues v.n - c, v.n (d times), v.n + c, c^2 = gamma p / rho."""
    rng = np.random.default_rng(7)
    ph = Physics(1.4, 1.0, 0.72, 0.5)
    u, _ = rand_state(rng, dim, n=3)
    for k in range(3):
        n = rng.normal(size=dim)
        n /= np.linalg.norm(n)
        A = np.zeros((dim + 2, dim + 2))
        for b in range(dim + 2):
            du = np.zeros(dim + 2)
            du[b] = 1e-30
            A[:, b] = (convective_flux(u[k] + 1j * du, ph) @ n).imag / 1e-30
        rho, v, E, p = primitives(u[k], 1.4)
        c = np.sqrt(1.4 * p / rho)
        vn = v @ n
        ev = np.sort(np.linalg.eigvals(A).real)
        assert np.allclose(ev, np.sort([vn - c] + [vn] * dim + [vn + c]), atol=1e-10)


def test_numerical_flux_is_local_lax_friedrichs():
    """With q = 0 and uhat the average of two states, the HDG flux seen from the
    left equals the local Lax-Friedrichs flux 1/2 (F(uL) + F(uR)).n + tau/2 (uL - uR)
    up to O(|uL - uR|^2)."""
    from oracle.physics import numerical_flux
    rng = np.random.default_rng(8)
    ph = Physics(1.4, 10.0, 0.72, 0.5)
    uL, _ = rand_state(rng, 3, n=1)
    delta = 1e-4 * rng.normal(size=uL.shape)
    uR = uL + delta
    n = np.array([0.6, 0.0, 0.8])
    q = np.zeros((1, 5, 3))
    tau = 3.0
    fh = numerical_flux(uL, 0.5 * (uL + uR), q, None, n, tau, ph)
    lf = 0.5 * (convective_flux(uL, ph) + convective_flux(uR, ph)) @ n + 0.5 * tau * (uL - uR)
    assert np.abs(fh - lf).max() < 1e-2 * np.abs(tau * delta).max()   # O(delta^2) gap only
