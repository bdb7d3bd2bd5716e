"""Reduced-basis initial guess for the condensed trace solve, in plain FP64.

Oracle (test infrastructure only).  Follows Sec. 3.4, eq. rb-min: a window
of at most nb_max previously accepted trace corrections W = [w_1 .. w_nb]
and their stored products Z = [S w_1 .. S w_nb] (each product taken with the
trace operator current when its column was inserted); the initial guess for
the system S dUhat = g is W c with c = argmin ||g - Z c||_2.  Inserting into
a full window discards the oldest column.  The least-squares problem is
solved with numpy's SVD-based lstsq (minimum-norm solution; singular values
below rcond * the largest are treated as zero).
"""
from __future__ import annotations

from collections import deque

import numpy as np


class ReducedBasis:
    def __init__(self, nb_max: int, rcond: float = 1e-12):
        self.nb_max = nb_max
        self.rcond = rcond
        self.W = deque(maxlen=nb_max)
        self.Z = deque(maxlen=nb_max)

    def push(self, w, z):
        """Insert an accepted correction w and its product z = S w."""
        self.W.append(np.array(w, dtype=float).ravel())
        self.Z.append(np.array(z, dtype=float).ravel())

    def coefficients(self, g):
        if not self.Z:
            return np.zeros(0)
        Z = np.stack(self.Z, axis=1)
        c, *_ = np.linalg.lstsq(Z, np.ravel(g), rcond=self.rcond)
        return c

    def guess(self, g):
        """dUhat_0 = W c (zero when the window is empty)."""
        c = self.coefficients(g)
        if c.size == 0:
            return np.zeros(np.size(g))
        return np.stack(self.W, axis=1) @ c
