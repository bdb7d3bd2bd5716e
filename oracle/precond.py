"""Trace-space preconditioners, in plain FP64.

Oracle (test infrastructure only).  Follows Sec. 3.3, eq. additive-schwarz:
the one-level additive Schwarz preconditioner on element-centred face patches,

    M_AS^{-1} = sum_r R_r^T S_r^{-1} R_r,   S_r = R_r S R_r^T,

where R_r is the 0/1 restriction from the global trace vector onto the trace
unknowns of the nf faces of element r (faces in local order, each face's
block of m * Nfp unknowns in the face's canonical order).  No coarse space.
Block-Jacobi (one patch per face) is the special case used as the default
preconditioner.  Everything is formed densely from the definition.
"""
from __future__ import annotations

import numpy as np


def restriction(conn, e: int, bs: int) -> np.ndarray:
    """R_r for element e: [nf * bs][F * bs] with one 1 per row."""
    nf = conn.e2f.shape[1]
    R = np.zeros((nf * bs, conn.n_faces * bs))
    for f in range(nf):
        F = int(conn.e2f[e, f])
        R[f * bs:(f + 1) * bs, F * bs:(F + 1) * bs] = np.eye(bs)
    return R


def additive_schwarz_matrix(S: np.ndarray, conn, bs: int) -> np.ndarray:
    """The dense matrix M_AS^{-1} of eq. additive-schwarz."""
    Minv = np.zeros_like(S)
    for e in range(conn.e2f.shape[0]):
        R = restriction(conn, e, bs)
        Sr = R @ S @ R.T
        Minv += R.T @ np.linalg.inv(Sr) @ R
    return Minv


def block_jacobi_matrix(S: np.ndarray, n_faces: int, bs: int) -> np.ndarray:
    """Inverse of the block diagonal of S (one block per face)."""
    Minv = np.zeros_like(S)
    for F in range(n_faces):
        sl = slice(F * bs, (F + 1) * bs)
        Minv[sl, sl] = np.linalg.inv(S[sl, sl])
    return Minv


def additive_schwarz_matrix_offsets(S: np.ndarray, e2f: np.ndarray, hoff: np.ndarray) -> np.ndarray:
    """M_AS^{-1} of eq. additive-schwarz when face blocks differ in size (tetrahedra
    of mixed degree): face F owns the trace unknowns hoff[F] .. hoff[F+1] - 1, and
    the patch of element e is the concatenation of its faces e2f[e] in local order."""
    Minv = np.zeros_like(S)
    for faces in e2f:
        idx = np.concatenate([np.arange(hoff[F], hoff[F + 1]) for F in faces])
        Sr = S[np.ix_(idx, idx)]                      # R_r S R_r^T
        Minv[np.ix_(idx, idx)] += np.linalg.inv(Sr)   # R_r^T S_r^{-1} R_r
    return Minv
