"""Pins of the oracle's reference element against closed forms (no GPU)."""
import itertools
import math

import numpy as np
import pytest

from oracle.refelem import RefElem, gauss_rule, gll_nodes, lagrange, lagrange_deriv


def mono_int(n):
    """Closed form of the integral of x^n over [-1, 1]."""
    return 0.0 if n % 2 else 2.0 / (n + 1)


def test_gll_closed_forms():
    assert np.allclose(gll_nodes(1), [-1, 1])
    assert np.allclose(gll_nodes(2), [-1, 0, 1])
    a = 1 / math.sqrt(5)
    assert np.allclose(gll_nodes(3), [-1, -a, a, 1], atol=1e-15)
    b = math.sqrt(3 / 7)
    assert np.allclose(gll_nodes(4), [-1, -b, 0, b, 1], atol=1e-15)


def test_gauss_closed_forms():
    x, w = gauss_rule(2)
    assert np.allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)]) and np.allclose(w, [1, 1])
    x, w = gauss_rule(3)
    assert np.allclose(x, [-math.sqrt(0.6), 0, math.sqrt(0.6)])
    assert np.allclose(w, [5 / 9, 8 / 9, 5 / 9])


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2), (3, 3)])
def test_quadrature_exact_on_monomials(d, p):
    """Tensor Gauss with p+2 points integrates x^a y^b (z^c) exactly, a,b,c <= 2p+3."""
    r = RefElem(d, p)
    for pw in itertools.product(range(2 * p + 4), repeat=d):
        vals = np.prod([r.xq[:, k] ** pw[k] for k in range(d)], axis=0)
        exact = np.prod([mono_int(n) for n in pw])
        assert abs(vals @ r.wq - exact) < 1e-13
    # face rule
    for pw in itertools.product(range(2 * p + 4), repeat=d - 1):
        f = 0
        others = [k for k in range(d) if k != 0]
        vals = np.prod([r.xf[f, :, others[a]] ** pw[a] for a in range(d - 1)], axis=0)
        exact = np.prod([mono_int(n) for n in pw])
        assert abs(vals @ r.wf - exact) < 1e-13


@pytest.mark.parametrize("d,p", [(2, 2), (3, 2), (3, 3)])
def test_basis_partition_and_derivatives(d, p):
    r = RefElem(d, p)
    assert np.allclose(r.phi.sum(1), 1.0, atol=1e-14)
    assert np.allclose(r.dphi.sum(2), 0.0, atol=1e-12)
    # derivatives of an interpolated degree-p polynomial are exact
    nodes = np.array([[r.nodes1[(j // r.n1 ** k) % r.n1] for k in range(d)] for j in range(r.Np)])
    rng = np.random.default_rng(0)
    for _ in range(5):
        pw = rng.integers(0, p + 1, size=d)
        f = np.prod([nodes[:, k] ** pw[k] for k in range(d)], axis=0)
        for k in range(d):
            exact = pw[k] * r.xq[:, k] ** max(pw[k] - 1, 0) * np.prod(
                [r.xq[:, kk] ** pw[kk] for kk in range(d) if kk != k], axis=0)
            if pw[k] == 0:
                exact = np.zeros(r.Nq)
            assert np.allclose(r.dphi[k] @ f, exact, atol=1e-12)


def test_lagrange_cardinal_and_derivative():
    x = gll_nodes(4)
    assert np.allclose(lagrange(x, x), np.eye(5), atol=1e-14)
    # derivative of interpolated x^3 equals 3 x^2
    pts = np.linspace(-1, 1, 7)
    assert np.allclose(lagrange_deriv(x, pts) @ (x ** 3), 3 * pts ** 2, atol=1e-12)


@pytest.mark.parametrize("d,p", [(2, 2), (3, 2), (3, 3)])
def test_face_trace_is_face_lagrange(d, p):
    """On GLL nodes the element basis restricted to face f is the face basis."""
    r = RefElem(d, p)
    for f in range(r.nf):
        assert np.allclose(r.phif[f][:, r.fnode[f]], r.mu, atol=1e-14)
        others = np.setdiff1d(np.arange(r.Np), r.fnode[f])
        assert np.allclose(r.phif[f][:, others], 0.0, atol=1e-14)
