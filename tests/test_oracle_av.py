"""The oracle's artificial-viscosity sensor, smoothing and TGV diagnostics
against closed forms.

* Sensor: zero for a uniform state, a pure expansion and a rigid rotation;
  for a linear compression v = -a x (uniform rho, p) it equals
  c_av min(sqrt(h/k) d a / c, s_max); with an added rotation the Ducros factor
  (d a)^2 / ((d a)^2 + omega^2) appears exactly (2-D: omega = 2 Omega).
* Smoothing: constants are preserved; the first pass of an isolated unit
  value on a uniform periodic mesh puts 1/2^d on its own vertices only; every
  pass preserves the vertex sum on a uniform periodic mesh; multilinear
  interpolation reproduces a linear vertex field exactly.
* Diagnostics: for v = A x with uniform rho and T on a box, E_k, eps_S and
  eps_D equal their integrals in closed form; for the TGV initial state on a
  fine mesh, E_k -> 1/8, eps_S -> 3/(4 Re) mu~(1) and eps_D -> 0.
"""
import numpy as np
import pytest

import synth
from oracle.av import (av_field, interpolate_q1, nodal_sensor, smooth, tgv_diagnostics)
from oracle.refelem import RefElem


def linear_velocity_state(mesh, p, A, gamma=1.4, mach=0.5):
    """rho = 1, p = p_inf uniform, v = A x: nodal U and exact Q."""
    d = mesh.dim
    x = synth.node_xyz(mesh, p)                     # [E][Np][d]
    v = np.einsum("ij,enj->eni", A, x)
    pinf = 1.0 / (gamma * mach ** 2)
    E = pinf / (gamma - 1) + 0.5 * np.sum(v * v, -1)
    u = np.concatenate([np.ones(x.shape[:2] + (1,)), v, E[..., None]], -1)   # [E][Np][m]
    # q_{a,j} = d_j u_a: rho const; d_j (rho v_i) = A_ij; d_j (rho E) = v_i A_ij
    q = np.zeros(x.shape[:2] + (d, d + 2))
    for j in range(d):
        for i in range(d):
            q[..., j, 1 + i] = A[i, j]
        q[..., j, d + 1] = np.einsum("eni,i->en", v, A[:, j])
    U = np.ascontiguousarray(u.transpose(0, 2, 1))
    Q = np.ascontiguousarray(q.transpose(0, 2, 3, 1))
    return U, Q, pinf


@pytest.mark.parametrize("dim", [2, 3])
def test_sensor_closed_forms(dim):
    gamma = 1.4
    mesh = synth.box_mesh(dim, (3,) * dim, (0,) * dim, (1,) * dim, (False,) * dim)
    p, c_av, h, smax = 2, 0.7, 0.1, 10.0
    I = np.eye(dim)
    for A in (0 * I, 0.3 * I):                      # uniform, expansion
        U, Q, _ = linear_velocity_state(mesh, p, A)
        assert np.abs(nodal_sensor(U, Q, gamma, c_av, h, p, smax)).max() == 0.0
    R = np.zeros((dim, dim)); R[0, 1], R[1, 0] = -0.4, 0.4
    U, Q, _ = linear_velocity_state(mesh, p, R)     # rigid rotation
    assert np.abs(nodal_sensor(U, Q, gamma, c_av, h, p, smax)).max() < 1e-14
    a = 0.25
    U, Q, pinf = linear_velocity_state(mesh, p, -a * I)
    c = np.sqrt(gamma * pinf)                      # rho = 1
    s = nodal_sensor(U, Q, gamma, c_av, h, p, smax)
    assert np.allclose(s, c_av * min(np.sqrt(h / p) * dim * a / c, smax), rtol=1e-12)
    s = nodal_sensor(U, Q, gamma, c_av, h, p, 0.01)  # clamped
    assert np.allclose(s, c_av * 0.01, rtol=1e-12)
    U, Q, pinf = linear_velocity_state(mesh, p, -a * I + R)
    om = 0.8                                        # |curl| of the rotation part
    duc = (dim * a) ** 2 / ((dim * a) ** 2 + om ** 2)
    s = nodal_sensor(U, Q, gamma, c_av, h, p, smax)
    assert np.allclose(s, c_av * np.sqrt(h / p) * dim * a / c * duc, rtol=1e-10)


@pytest.mark.parametrize("dim", [2, 3])
def test_smoothing_closed_forms(dim):
    mesh = synth.box_mesh(dim, (4,) * dim, (0,) * dim, (1,) * dim, (True,) * dim)
    E = mesh.n_elem
    nv = smooth(mesh, np.full(E, 2.5))
    used = np.unique(mesh.periodic_map[mesh.elem_vert])
    assert np.allclose(nv[used], 2.5)
    delta = np.zeros(E)
    delta[5] = 1.0
    v1 = smooth(mesh, delta, passes=1)
    own = set(mesh.periodic_map[mesh.elem_vert[5]])
    for v in used:
        assert v1[v] == (1.0 / 2 ** dim if v in own else 0.0)
    for passes in (1, 2, 3):
        assert abs(smooth(mesh, delta, passes)[used].sum() - 1.0) < 1e-14
    # multilinear interpolation reproduces a linear field (non-periodic mesh)
    m2 = synth.box_mesh(dim, (3,) * dim, (0,) * dim, (2.0,) * dim, (False,) * dim)
    lin = m2.vert_xyz @ np.arange(1, dim + 1) + 0.5
    ref = RefElem(dim, 3)
    out = interpolate_q1(m2, 3, lin, ref.nodes1)
    x = synth.node_xyz(m2, 3)
    assert np.allclose(out, x @ np.arange(1, dim + 1) + 0.5, atol=1e-13)


def test_diagnostics_linear_field():
    dim = 3
    mesh = synth.box_mesh(dim, (3, 3, 3), (0,) * 3, (1.0, 2.0, 1.5), (False,) * 3)
    P = synth.tiny(3, 2, periodic=False)
    P.mesh = mesh
    A = np.array([[0.1, -0.3, 0.0], [0.3, -0.2, 0.1], [0.0, 0.2, 0.05]])
    U, Q, _ = linear_velocity_state(mesh, 2, A, gamma=P.gamma, mach=P.mach)
    P.visc_law = 0
    Ek, eS, eD, vol = tgv_diagnostics(P, U, Q)
    L = np.array([1.0, 2.0, 1.5])
    assert abs(vol - L.prod()) < 1e-12
    # int |A x|^2 over the box [0,L]: sum_i sum_jk A_ij A_ik int x_j x_k
    M2 = np.outer(L / 2, L / 2)
    np.fill_diagonal(M2, L ** 2 / 3)
    Ek_ref = 0.5 * np.einsum("ij,ik,jk->", A, A, M2)
    om = np.array([A[2, 1] - A[1, 2], A[0, 2] - A[2, 0], A[1, 0] - A[0, 1]])
    assert abs(Ek - Ek_ref) < 1e-12
    assert abs(eS - om @ om / P.re) < 1e-12
    assert abs(eD - 4 / 3 * np.trace(A) ** 2 / P.re) < 1e-12


@pytest.mark.parametrize("law", [0, 1])
def test_diagnostics_tgv_initial_state(law):
    P = synth.config_tgv(6, 3, 0.1, 0, False, 0.0)
    P.visc_law = law
    Ek, eS, eD, vol = tgv_diagnostics(P, P.U, P.Q)
    mu1 = 1.0 if law == 0 else P.suth_c1 / (1.0 + P.suth_s)
    assert abs(vol - (2 * np.pi) ** 3) < 1e-9
    assert abs(Ek - 0.125) < 2e-5
    assert abs(eS - 0.75 * mu1 / P.re) < 2e-3 * 0.75 / P.re
    assert abs(eD) < 1e-4 * 0.75 / P.re


def test_av_field_is_nonnegative_and_bounded():
    P = synth.config_tgv(4, 2, 1.25, 2, False, 0.0)
    ref = RefElem(3, 2)
    nu = av_field(P, P.U, P.Q, c_av=2e-3, h_m=2 * np.pi / 4, s_max=1.0, nodes1=ref.nodes1)
    assert nu.shape == P.U[:, 0, :].shape
    assert nu.min() >= 0.0 and nu.max() <= 2e-3 + 1e-18
