"""The oracle's reduced-basis initial guess against closed forms.

* If g lies in span(Z) with full column rank, the minimiser is exact:
  g = Z c*  gives  c = c*  and  W c = W c*.
* With a fixed operator S and columns w_i solving S w_i = g_i, any g that is
  a combination of the g_i is solved exactly by the guess.
* The guess never has a larger residual than the zero guess, and its residual
  is orthogonal to span(Z) (normal equations).
* The window keeps the nb_max most recent columns.
"""
import numpy as np

from oracle.rb import ReducedBasis


def test_exact_in_span():
    rng = np.random.default_rng(0)
    n, k = 200, 6
    W = rng.normal(size=(n, k))
    Z = rng.normal(size=(n, k))
    rb = ReducedBasis(8)
    for i in range(k):
        rb.push(W[:, i], Z[:, i])
    cs = rng.normal(size=k)
    assert np.allclose(rb.coefficients(Z @ cs), cs, rtol=1e-12, atol=1e-12)
    assert np.allclose(rb.guess(Z @ cs), W @ cs, rtol=1e-12, atol=1e-12)


def test_previous_solutions_reproduce_combinations():
    rng = np.random.default_rng(1)
    n = 60
    S = rng.normal(size=(n, n)) + 8 * np.eye(n)
    rb = ReducedBasis(5)
    G = rng.normal(size=(n, 5))
    for i in range(5):
        w = np.linalg.solve(S, G[:, i])
        rb.push(w, S @ w)
    g = G @ np.array([0.3, -1.0, 2.0, 0.0, 0.5])
    assert np.allclose(rb.guess(g), np.linalg.solve(S, g), rtol=1e-10, atol=1e-12)


def test_residual_not_worse_and_orthogonal():
    rng = np.random.default_rng(2)
    n = 100
    rb = ReducedBasis(4)
    for _ in range(4):
        rb.push(rng.normal(size=n), rng.normal(size=n))
    g = rng.normal(size=n)
    Z = np.stack(rb.Z, axis=1)
    r = g - Z @ rb.coefficients(g)
    assert np.linalg.norm(r) <= np.linalg.norm(g)
    assert np.abs(Z.T @ r).max() < 1e-12 * np.linalg.norm(g) * np.abs(Z).max() * n


def test_window_drops_oldest():
    rb = ReducedBasis(3)
    for i in range(5):
        rb.push(np.full(4, float(i)), np.eye(4)[i % 4])
    assert [w[0] for w in rb.W] == [2.0, 3.0, 4.0]
    assert len(rb.Z) == 3 and rb.guess(np.zeros(4)).shape == (4,)
    assert np.array_equal(ReducedBasis(2).guess(np.ones(3)), np.zeros(3))
