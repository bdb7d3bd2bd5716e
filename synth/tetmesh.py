"""Seeded tetrahedral meshes of mixed degree on quadratic geometry.

Inputs only (no method arithmetic): a structured box of hexahedral cells, each
split into six Kuhn tetrahedra along its main diagonal, vertices placed by a
wall-normal graded coordinate and an optional wall bump, quadratic (10-node)
element geometry, a seeded per-element degree, and nodal states sampled at
the element nodes.

Conventions (the data interface of the library's tetrahedral path):

* element vertices ``elem_vert [E][4]`` with positive orientation (the
  reference tetrahedron v0 = (-1,-1,-1), v1 = (1,-1,-1), v2 = (-1,1,-1),
  v3 = (-1,-1,1) maps with det J > 0); local face f is opposite vertex f;
* ``geo [E][10][3]``: the 4 vertices, then the midpoints of edges 01, 02, 03,
  12, 13, 23; a midpoint is the bump image of the straight midpoint when the
  edge is curved, else the average of its end points;
* element nodes: the equispaced lattice (i, j, k), i + j + k <= p, k slowest,
  mapped by the quadratic geometry;
* packed state: ``U`` = per element [m][Np_e] back to back, ``Q`` = per
  element [3][m][Np_e], ``UH`` = per face [m][Nfp_F] back to back.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

from . import conserved, freestream, graded_coordinates, normal, uniform

EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


@dataclass
class TetMesh:
    vert_xyz: np.ndarray       # [n_vert][3]
    elem_vert: np.ndarray      # [E][4] int64
    periodic_map: np.ndarray   # [n_vert] int64
    bnd_tag: np.ndarray        # [E][4] int32
    elem_p: np.ndarray         # [E] int32
    geo: np.ndarray            # [E][10][3]
    n: tuple = ()

    @property
    def n_elem(self) -> int:
        return int(self.elem_vert.shape[0])


def _orient(X):
    J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
    return np.linalg.det(J)


def kuhn_box(n, coords, periodic, tags=None, degrees=None, bump=None, curved_layers=0, seed=3, pmax=4):
    """Structured box of n = (nx, ny, nz) cells, six tetrahedra per cell.

    ``coords``: per-direction vertex coordinates (length n_r + 1).  ``tags``
    maps a box side (r, s) to a boundary tag (default 1).  ``degrees``: a
    fixed degree, or None for a seeded uniform draw in 1..pmax.  ``bump(x)``
    maps computational to physical points ([k, 3] -> [k, 3]); edges whose two
    end points lie in the first ``curved_layers`` cell layers above y = 0 get
    the bump image of their midpoint, the others a straight midpoint.
    """
    n = tuple(int(v) for v in n)
    nv = [n[r] + 1 for r in range(3)]
    tags = tags or {}
    for r in range(3):
        if periodic[r] and n[r] < 3:
            raise ValueError("periodic directions need at least 3 cells")

    def vid(i, j, k):
        return i + nv[0] * (j + nv[1] * k)

    comp = np.array([[coords[0][i], coords[1][j], coords[2][k]]
                     for k in range(nv[2]) for j in range(nv[1]) for i in range(nv[0])])
    phys = comp if bump is None else bump(comp)
    pmap = np.arange(comp.shape[0], dtype=np.int64)
    for k in range(nv[2]):
        for j in range(nv[1]):
            for i in range(nv[0]):
                ii = [i, j, k]
                jj = [0 if (periodic[r] and ii[r] == n[r]) else ii[r] for r in range(3)]
                pmap[vid(i, j, k)] = vid(*jj)
    ev, tag, rows = [], [], []
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                for perm in itertools.permutations(range(3)):
                    c = [0, 0, 0]
                    cs = [tuple(c)]
                    for r in perm[:2]:
                        c[r] = 1
                        cs.append(tuple(c))
                    cs.append((1, 1, 1))
                    ids = [vid(i + a, j + b, k + cc) for (a, b, cc) in cs]
                    if _orient(phys[ids]) < 0:
                        ids[1], ids[2] = ids[2], ids[1]
                        cs[1], cs[2] = cs[2], cs[1]
                    ev.append(ids)
                    rows.append([j + q[1] for q in cs])
                    cell = (i, j, k)
                    t = []
                    for f in range(4):
                        loc = [cs[v] for v in range(4) if v != f]
                        tf = 0
                        for r in range(3):
                            for s in (0, 1):
                                if periodic[r]:
                                    continue
                                side = 0 if s == 0 else n[r]
                                if all(cell[r] + q[r] == side for q in loc):
                                    tf = tags.get((r, s), 1)
                        t.append(tf)
                    tag.append(t)
    evv = np.array(ev, dtype=np.int64)
    rows = np.array(rows)
    geo = np.zeros((evv.shape[0], 10, 3))
    geo[:, :4] = phys[evv]
    for c, (a, b) in enumerate(EDGES):
        straight = 0.5 * (phys[evv[:, a]] + phys[evv[:, b]])
        if bump is None:
            geo[:, 4 + c] = straight
            continue
        bent = bump(0.5 * (comp[evv[:, a]] + comp[evv[:, b]]))
        curved = np.maximum(rows[:, a], rows[:, b]) <= curved_layers
        geo[:, 4 + c] = np.where(curved[:, None], bent, straight)
    ev = np.array(ev, dtype=np.int64)
    E = ev.shape[0]
    if degrees is None:
        elem_p = (1 + np.floor(pmax * uniform(seed, E))).astype(np.int32)
    else:
        elem_p = np.full(E, int(degrees), dtype=np.int32)
    return TetMesh(phys.astype(np.float64), ev, pmap, np.array(tag, dtype=np.int32), elem_p, geo, n)


def lattice(p):
    return [(i, j, k) for k in range(p + 1) for j in range(p + 1 - k) for i in range(p + 1 - j - k)]


def node_shape(p):
    """Quadratic shape functions at the degree-p lattice: [Np][10]."""
    out = []
    for (i, j, k) in lattice(p):
        l1, l2, l3 = i / p, j / p, k / p
        lam = [1.0 - l1 - l2 - l3, l1, l2, l3]
        out.append([lam[v] * (2 * lam[v] - 1) for v in range(4)] + [4 * lam[a] * lam[b] for (a, b) in EDGES])
    return np.array(out)


def node_xyz(mesh: TetMesh, e: int) -> np.ndarray:
    """Physical positions [Np][3] of element e's nodes (quadratic geometry)."""
    p = int(mesh.elem_p[e])
    out = []
    for (i, j, k) in lattice(p):
        l1, l2, l3 = i / p, j / p, k / p
        lam = [1.0 - l1 - l2 - l3, l1, l2, l3]
        N = [lam[v] * (2 * lam[v] - 1) for v in range(4)] + [4 * lam[a] * lam[b] for (a, b) in EDGES]
        out.append(np.asarray(N) @ mesh.geo[e])
    return np.array(out)


def wall_bump(amp=0.05):
    """y <- y + amp sin(pi x) (1 - y)^2."""
    def f(x):
        x = np.array(x, dtype=float, copy=True)
        x[:, 1] = x[:, 1] + amp * np.sin(np.pi * x[:, 0]) * (1.0 - x[:, 1]) ** 2
        return x
    return f


def sinusoids(gamma, mach, seed, amp, axes=3):
    """Freestream along x plus amp * sum of 4 seeded sinusoids in rho, rho u, rho E."""
    r = uniform(seed, 12)
    ab = 1 + np.floor(3 * r[:8]).astype(int)
    ph = 2 * np.pi * r[8:12]

    def fun(x):
        ub = freestream(3, gamma, mach)
        u = np.broadcast_to(ub, x.shape[:-1] + (5,)).copy()
        s = np.zeros(x.shape[:-1])
        for k in range(4):
            s = s + np.sin(2 * np.pi * (ab[2 * k] * x[..., 0] + ab[2 * k + 1] * x[..., 2]) + ph[k])
        for a in (0, 1, 4):
            u[..., a] = u[..., a] + amp * s
        return u
    return fun


def packed_state(mesh: TetMesh, fun, face_nfp, ubg, seed, noise=1e-4, trace_noise=1e-3, q_noise=1e-2):
    """U, Q, UH, Ustar packed as in the module docstring.

    U samples ``fun`` at the element nodes plus seeded noise; Q is seeded noise
    of size q_noise (any Q is admissible for a linearization); UH is the
    background state ubg plus relative noise, one [m][Nfp] block per face with
    the sizes ``face_nfp``.
    """
    U = [None] * mesh.n_elem
    for p in np.unique(mesh.elem_p):
        idx = np.nonzero(mesh.elem_p == p)[0]
        x = np.einsum("nc,eck->enk", node_shape(int(p)), mesh.geo[idx])       # [E_p][Np][3]
        u = fun(x)                                                             # [E_p][Np][m]
        for r, e in enumerate(idx):
            U[e] = u[r].T.ravel()
    U = np.concatenate(U)
    U = U + noise * normal(seed, U.size)
    Q = q_noise * normal(seed + 1, 3 * U.size)
    UH = np.concatenate([np.repeat(ubg, int(k)) for k in face_nfp])
    scale = np.concatenate([np.repeat(np.abs(ubg) + 1.0, int(k)) for k in face_nfp])
    UH = UH + trace_noise * scale * normal(seed + 2, UH.size)
    return U, Q, UH, U.copy()


@dataclass
class TetProblem:
    name: str
    mesh: TetMesh
    gamma: float
    re: float
    pr: float
    mach: float
    tau: float
    dt: float
    a_ii: float
    visc_law: int
    suth_c1: float
    suth_s: float
    ubc: np.ndarray
    twall: float = 1.0


def config4_mesh(nx=30, ny=20, nz=28, ratio=1.2, aspect=1e3, curved_layers=None, seed=3, degrees=None):
    """Curved anisotropic wall layer: x in [0, 1] and z in [0, nz / nx] periodic,
    y graded from the wall (first cell dx / aspect, growth ratio), adiabatic
    wall at y = 0 (tag 4), far field on top (tag 1), bump y += 0.05 sin(pi x)(1 - y)^2."""
    dx = 1.0 / nx
    h1 = dx / aspect
    ys = np.concatenate([[0.0], np.cumsum(h1 * ratio ** np.arange(ny))])
    coords = [np.linspace(0.0, 1.0, nx + 1), ys, np.linspace(0.0, nz * dx, nz + 1)]
    # curved wall layer: edges become straight only above the first cell layer whose height is six
    # times the bump's sagitta over one cell (0.05 pi^2 dx^2 / 8), so that the quadratic elements of
    # the transition stay valid (14 of 20 layers for nx = 30)
    if curved_layers is None:
        sag = 0.05 * np.pi ** 2 * dx * dx / 8.0
        cl = next((j for j in range(ny) if h1 * ratio ** j >= 6.0 * sag), ny)
    else:
        cl = curved_layers
    return kuhn_box((nx, ny, nz), coords, (True, False, True), tags={(1, 0): 4, (1, 1): 1}, degrees=degrees,
                    bump=wall_bump(0.05), curved_layers=cl, seed=seed)


def config4_problem(mesh: TetMesh, mach=0.5, re=1e5, gamma=1.4, pr=0.72):
    return TetProblem("tet-mixed-p-curved", mesh, gamma, re, pr, mach, tau=5.0, dt=1e-3, a_ii=0.4358665215,
                      visc_law=0, suth_c1=1.0, suth_s=0.0, ubc=freestream(3, gamma, mach))


__all__ = ["TetMesh", "kuhn_box", "node_xyz", "wall_bump", "sinusoids", "packed_state", "TetProblem",
           "config4_mesh", "config4_problem", "conserved", "graded_coordinates"]
