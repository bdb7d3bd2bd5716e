"""The oracle's additive Schwarz preconditioner against closed forms.

* A block-diagonal operator (one dense block per face): every patch solve
  inverts the blocks of its faces, so M^{-1} x on face F is n_F S_FF^{-1} x_F,
  n_F = number of elements that share F (2 inside, 1 on a boundary face).
* Symmetric S gives a symmetric M^{-1}, and for SPD S the preconditioned
  operator M^{-1} S has real positive eigenvalues.
* Block-Jacobi inverts a block-diagonal operator exactly, and on a periodic
  mesh (every face in two patches) the Schwarz operator is twice that.
"""
import numpy as np
import pytest

import synth
from oracle.mesh import Connectivity
from oracle.precond import additive_schwarz_matrix, block_jacobi_matrix


def pattern_matrix(conn, bs, rng, spd=False, diag_only=False):
    F = conn.n_faces
    S = np.zeros((F * bs, F * bs))
    for f in range(F):
        for b in range(conn.rowptr[f], conn.rowptr[f + 1]):
            g = conn.col[b]
            if diag_only and g != f:
                continue
            S[f * bs:(f + 1) * bs, g * bs:(g + 1) * bs] = rng.normal(size=(bs, bs))
    if spd:
        S = S + S.T
        # diagonal shift keeps the pattern and makes S SPD
        S += (np.abs(np.linalg.eigvalsh(S)).max() + 1.0) * np.eye(F * bs)
    else:
        S += 4 * bs * np.eye(F * bs)
    return S


@pytest.mark.parametrize("per", [True, (True, False)], ids=["periodic", "boundary"])
def test_block_diagonal_operator_closed_form(per):
    mesh = synth.box_mesh(2, (3, 4), (0, 0), (1, 1), per if isinstance(per, tuple) else (True, True))
    conn = Connectivity(mesh, 2)
    bs = 4 * 3
    rng = np.random.default_rng(0)
    S = pattern_matrix(conn, bs, rng, diag_only=True)
    M = additive_schwarz_matrix(S, conn, bs)
    x = rng.normal(size=conn.n_faces * bs)
    y = M @ x
    nF = (conn.f2e[:, :, 0] >= 0).sum(axis=1)
    assert (nF == 1).any() == (per is not True)
    for F in range(conn.n_faces):
        sl = slice(F * bs, (F + 1) * bs)
        ref = nF[F] * np.linalg.solve(S[sl, sl], x[sl])
        assert np.allclose(y[sl], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_symmetry_and_positive_spectrum():
    mesh = synth.box_mesh(2, (3, 3), (0, 0), (1, 1), (True, True))
    conn = Connectivity(mesh, 1)
    bs = 4 * 2
    S = pattern_matrix(conn, bs, np.random.default_rng(1), spd=True)
    M = additive_schwarz_matrix(S, conn, bs)
    assert np.abs(M - M.T).max() < 1e-12 * np.abs(M).max()
    ev = np.linalg.eigvals(M @ S)
    assert np.abs(ev.imag).max() < 1e-8 and ev.real.min() > 0


def test_block_jacobi_is_exact_on_block_diagonal_operator():
    mesh = synth.box_mesh(3, (3, 3, 3), (0,) * 3, (1,) * 3, (True,) * 3)
    conn = Connectivity(mesh, 1)
    bs = 5 * 4
    S = pattern_matrix(conn, bs, np.random.default_rng(2), diag_only=True)
    assert np.allclose(block_jacobi_matrix(S, conn.n_faces, bs) @ S, np.eye(S.shape[0]), atol=1e-12)
    # and the additive Schwarz operator is exactly twice that on a periodic mesh
    M = additive_schwarz_matrix(S, conn, bs)
    assert np.allclose(M @ S, 2 * np.eye(S.shape[0]), atol=1e-11)


def test_variable_block_schwarz_closed_form_and_uniform_case():
    """Faces of different sizes (tetrahedra of mixed degree): on a block-diagonal
    operator the patch solves give n_F S_FF^{-1} x_F on every face; with equal
    sizes the variable-size form is the uniform one."""
    from oracle.precond import additive_schwarz_matrix_offsets
    from oracle.tet import TetConnectivity
    from synth import tetmesh as tm
    mesh = tm.kuhn_box((3, 1, 2), [np.linspace(0, 1, 4), np.linspace(0, .5, 2), np.linspace(0, .5, 3)],
                       (True, False, False), seed=3)
    conn = TetConnectivity(mesh)
    hoff = np.asarray(conn.hoff)
    sizes = np.diff(hoff)
    assert len(set(sizes.tolist())) > 1
    rng = np.random.default_rng(4)
    n = hoff[-1]
    S = np.zeros((n, n))
    for F in range(len(sizes)):
        sl = slice(hoff[F], hoff[F + 1])
        S[sl, sl] = rng.normal(size=(sizes[F], sizes[F])) + 3 * sizes[F] * np.eye(sizes[F])
    M = additive_schwarz_matrix_offsets(S, np.asarray(conn.e2f), hoff)
    x = rng.normal(size=n)
    y = M @ x
    nF = (np.asarray(conn.f2e)[:, :, 0] >= 0).sum(axis=1)
    assert (nF == 1).any() and (nF == 2).any()
    for F in range(len(sizes)):
        sl = slice(hoff[F], hoff[F + 1])
        ref = nF[F] * np.linalg.solve(S[sl, sl], x[sl])
        assert np.allclose(y[sl], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    # uniform sizes: the hex form
    mesh2 = synth.box_mesh(2, (3, 3), (0, 0), (1, 1), (True, True))
    c2 = Connectivity(mesh2, 1)
    bs = 4 * 2
    S2 = pattern_matrix(c2, bs, np.random.default_rng(5))
    h2 = np.arange(c2.n_faces + 1) * bs
    assert np.allclose(additive_schwarz_matrix_offsets(S2, c2.e2f, h2), additive_schwarz_matrix(S2, c2, bs),
                       rtol=0, atol=1e-12 * np.abs(S2).max())
