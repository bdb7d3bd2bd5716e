"""DIRK time stepping and Newton on the stage equations, in plain FP64.

Oracle (test infrastructure only).  Follows Sec. 2.3 (eqs. dirk-stage and
dirk-update) and the Newton iteration of Sec. 2.5 / 3.1:

* an s-stage DIRK method with Butcher matrix A (a_ij = 0 for j > i) and
  weights b; d = A^{-1}.  Stage i solves the stage equations whose mass term
  is sum_j d_ij M (U^{n,j} - U^n); dividing by d_ii = 1 / a_ii this is
  (1/a_ii) M (U^{n,i} - U*_i) with the known stage data
      U*_i = U^n - a_ii sum_{j<i} d_ij (U^{n,j} - U^n);
* the step ends with U^{n+1} = U^n + sum_j e_j (U^{n,j} - U^n),
  e_j = sum_i b_i d_ij;
* each stage is solved by Newton's method from the previous stage state: the
  condensed trace system is assembled and solved densely (numpy LU), the
  interior corrections are recovered element by element and the full
  correction is applied with unit step.

The Newton driver reuses oracle.hdg.Problem; nothing here runs on a GPU.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import brentq

from .hdg import Problem


def alexander_sdirk3():
    """Three-stage, third-order, L-stable, stiffly accurate SDIRK (Alexander 1977).

    The family has A = [[g, 0, 0], [c2 - g, g, 0], [b1, b2, g]],
    c = (g, c2, 1), c2 = (1 + g) / 2, b = last row of A.  For a given g the
    weights b1, b2 follow from the first two order conditions
    (sum b = 1, b.c = 1/2); g is the root in (0.4, 0.5) of the third
    (b.c^2 = 1/3).  The fourth condition, b.A.c = 1/6, and L-stability are
    checked by the tests, not imposed here.
    """
    def weights(g):
        c = np.array([g, (1.0 + g) / 2.0, 1.0])
        M = np.array([[1.0, 1.0], [c[0], c[1]]])
        rhs = np.array([1.0 - g, 0.5 - g * c[2]])
        b12 = np.linalg.solve(M, rhs)
        return np.array([b12[0], b12[1], g]), c

    def cond3(g):
        b, c = weights(g)
        return b @ (c * c) - 1.0 / 3.0

    g = brentq(cond3, 0.4, 0.5, xtol=1e-16, rtol=4 * np.finfo(float).eps, maxiter=200)
    b, c = weights(g)
    A = np.array([[g, 0.0, 0.0], [c[1] - g, g, 0.0], [b[0], b[1], g]])
    return A, b, c


def dirk_coefficients(A, b):
    """d = A^{-1} and e_j = sum_i b_i d_ij (eq. dirk-update)."""
    d = np.linalg.inv(np.asarray(A, float))
    e = np.asarray(b, float) @ d
    return d, e


def stage_data(Un, stages, A, d, i):
    """U*_i = U^n - a_ii sum_{j<i} d_ij (U^{n,j} - U^n)."""
    Us = np.array(Un, dtype=np.result_type(Un, 1.0), copy=True)
    for j in range(i):
        Us = Us - A[i][i] * d[i][j] * (stages[j] - Un)
    return Us


def dirk_step(solve_stage, Un, A, b):
    """One DIRK step with a caller-supplied stage solver.

    solve_stage(i, Ustar, a_ii) returns the stage state U^{n,i}; the result is
    (U^{n+1}, [U^{n,1}, ..., U^{n,s}]).
    """
    A = np.asarray(A, float)
    s = A.shape[0]
    d, e = dirk_coefficients(A, b)
    stages = []
    for i in range(s):
        Us = stage_data(Un, stages, A, d, i)
        stages.append(np.asarray(solve_stage(i, Us, A[i][i])))
    Unew = np.array(Un, dtype=np.result_type(Un, 1.0), copy=True)
    for j in range(s):
        Unew = Unew + e[j] * (stages[j] - Un)
    return Unew, stages


def dense_trace_matrix(vals, rowptr, col, bs):
    F = len(rowptr) - 1
    S = np.zeros((F * bs, F * bs))
    for f in range(F):
        for k in range(rowptr[f], rowptr[f + 1]):
            S[f * bs:(f + 1) * bs, col[k] * bs:(col[k] + 1) * bs] = vals[k]
    return S


def newton(pb: Problem, Q, U, UH, tol=1e-11, maxit=8, fixed=None):
    """Newton on the stage equations of pb (its Ustar, a_ii, dt).

    Stops when ||F|| <= tol, or after exactly `fixed` iterations when given.
    Returns (Q, U, UH, history of ||F|| before each iteration and at the end).
    """
    cn = pb.conn
    bs = pb.ref.m * pb.ref.Nfp
    Q, U, UH = (np.array(x, dtype=float, copy=True) for x in (Q, U, UH))
    hist = []
    nit = maxit if fixed is None else fixed
    for k in range(nit + 1):
        hist.append(pb.residual_norm(Q, U, UH))
        if k == nit or (fixed is None and hist[-1] <= tol):
            break
        pb.Q, pb.U, pb.UH = Q, U, UH
        vals, cache = pb.assemble()
        S = dense_trace_matrix(vals, cn.rowptr, cn.col, bs)
        gg = pb.assemble_g(cache, range(cn.n_faces))
        g = np.concatenate([gg[f].ravel() for f in range(cn.n_faces)])
        dUH = np.linalg.solve(S, g).reshape(UH.shape)
        dQ = np.zeros_like(Q)
        dU = np.zeros_like(U)
        for e in range(U.shape[0]):
            dQ[e], dU[e] = pb.recover(e, cache[e], dUH)
        Q, U, UH = Q + dQ, U + dU, UH + dUH
    return Q, U, UH, hist


def hdg_dirk_step(P, A, b, tol=1e-11, maxit=8, fixed=None):
    """One DIRK step of the HDG system from the state (P.Q, P.U, P.UH).

    Each stage starts Newton from the previous stage's (Q, U, Uhat).  For a
    stiffly accurate tableau (e = unit vector on the last stage) the returned
    Q and Uhat are the last stage's, consistent with U^{n+1}; otherwise the
    algebraic variables are those of the last stage and U^{n+1} is the
    combination of eq. dirk-update.
    Returns (Q, U^{n+1}, Uhat, stage histories).
    """
    pb = Problem(P)
    Un = np.array(P.U, dtype=float, copy=True)
    state = {"Q": np.array(P.Q, float), "U": Un.copy(), "UH": np.array(P.UH, float)}
    hists = []

    def solve_stage(i, Us, a_ii):
        pb.Ustar = Us
        pb.a_ii = a_ii
        Q, U, UH, h = newton(pb, state["Q"], state["U"], state["UH"], tol, maxit, fixed)
        state.update(Q=Q, U=U, UH=UH)
        hists.append(h)
        return U

    Unew, _ = dirk_step(solve_stage, Un, A, b)
    return state["Q"], Unew, state["UH"], hists
