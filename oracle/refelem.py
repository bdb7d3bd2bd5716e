"""Reference-element tables for tensor-product (quad / hex) HDG elements.

Oracle (test infrastructure only).  Spaces of Sec. 2.2 (eq. spaces) read as the
tensor space Q^k on [-1, 1]^d with nodal Lagrange bases on Gauss-Lobatto points;
integrals by tensor Gauss-Legendre rules with p + 2 points per direction
(exact to degree 2p + 3).  The trace basis of a face is the tensor Lagrange
basis on the face's own Gauss-Lobatto points.
"""
from __future__ import annotations

import itertools

import numpy as np
from numpy.polynomial import legendre as npleg


def gauss_rule(n: int):
    """n-point Gauss-Legendre rule on [-1, 1] (library routine)."""
    x, w = npleg.leggauss(n)
    return np.asarray(x, float), np.asarray(w, float)


def gll_nodes(p: int) -> np.ndarray:
    """Gauss-Lobatto nodes of degree p: -1, the roots of P_p', +1."""
    if p < 1:
        raise ValueError("p >= 1")
    c = np.zeros(p + 1)
    c[p] = 1.0
    inner = np.sort(npleg.legroots(npleg.legder(c)).real) if p > 1 else np.zeros(0)
    return np.concatenate([[-1.0], inner, [1.0]])


def lagrange(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Lagrange basis values ``L[k, j] = l_j(x_k)`` by the product formula."""
    n = len(nodes)
    out = np.ones((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                out[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return out


def lagrange_deriv(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Derivatives ``D[k, j] = l_j'(x_k)``: sum over the dropped factor."""
    n = len(nodes)
    out = np.zeros((len(x), n))
    for j in range(n):
        for m in range(n):
            if m == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[m]))
            for k in range(n):
                if k != j and k != m:
                    term = term * (x - nodes[k]) / (nodes[j] - nodes[k])
            out[:, j] += term
    return out


def tensor_index(idx, n):
    """Flat index of a multi-index, first direction fastest."""
    f = 0
    for r in reversed(range(len(idx))):
        f = f * n + idx[r]
    return f


class RefElem:
    """Tables of the reference quad (d = 2) or hex (d = 3) of degree p.

    Attributes (``g`` volume points, ``s`` face points, ``j`` element nodes,
    ``l`` face nodes in the face's local frame):

    * ``phi[g, j]``, ``dphi[r, g, j]`` (reference derivatives), ``wq[g]``;
    * ``xq[g, r]`` reference coordinates of volume points;
    * ``phif[f, s, j]``, ``dphif[f, r, s, j]`` element basis on face f;
    * ``xf[f, s, r]`` reference coordinates of face points, ``wf[s]``;
    * ``mu[s, l]`` trace basis at face points, ``fnode[f, l]`` element node of
      face node l;
    * ``nref[f]`` reference outward normal of face f.

    Local face ``f = 2 r + side``: the face ``xi_r = -1`` (side 0) or ``+1``
    (side 1); its local coordinates are the remaining directions in
    increasing order, the lower one fastest.
    """

    def __init__(self, d: int, p: int):
        self.d, self.p = d, p
        self.m = d + 2
        n1, q1 = p + 1, p + 2
        self.n1, self.q1 = n1, q1
        self.Np, self.Nq = n1 ** d, q1 ** d
        self.nf = 2 * d
        self.Nfp, self.Nfq = n1 ** (d - 1), q1 ** (d - 1)
        self.nodes1 = gll_nodes(p)
        xg, wg = gauss_rule(q1)
        B = lagrange(self.nodes1, xg)
        Dd = lagrange_deriv(self.nodes1, xg)
        # volume
        self.xq = np.zeros((self.Nq, d))
        self.wq = np.zeros(self.Nq)
        self.phi = np.zeros((self.Nq, self.Np))
        self.dphi = np.zeros((d, self.Nq, self.Np))
        for gi in itertools.product(range(q1), repeat=d):
            gi = tuple(reversed(gi))  # gi[0] fastest
            g = tensor_index(gi, q1)
            self.xq[g] = [xg[gi[r]] for r in range(d)]
            self.wq[g] = np.prod([wg[gi[r]] for r in range(d)])
            for jj in itertools.product(range(n1), repeat=d):
                jj = tuple(reversed(jj))
                j = tensor_index(jj, n1)
                self.phi[g, j] = np.prod([B[gi[r], jj[r]] for r in range(d)])
                for k in range(d):
                    self.dphi[k, g, j] = np.prod([(Dd if r == k else B)[gi[r], jj[r]] for r in range(d)])
        # faces
        self.wf = np.zeros(self.Nfq)
        self.xf = np.zeros((self.nf, self.Nfq, d))
        self.phif = np.zeros((self.nf, self.Nfq, self.Np))
        self.dphif = np.zeros((self.nf, d, self.Nfq, self.Np))
        self.fnode = np.zeros((self.nf, self.Nfp), dtype=np.int64)
        self.nref = np.zeros((self.nf, d))
        Bn = lagrange(self.nodes1, np.array([-1.0, 1.0]))
        Dn = lagrange_deriv(self.nodes1, np.array([-1.0, 1.0]))
        for f in range(self.nf):
            r, side = divmod(f, 2)
            others = [k for k in range(d) if k != r]
            self.nref[f, r] = -1.0 if side == 0 else 1.0
            for si in itertools.product(range(q1), repeat=d - 1):
                si = tuple(reversed(si))
                s = tensor_index(si, q1) if d > 1 else 0
                gi = [0] * d
                pt = [0.0] * d
                pt[r] = -1.0 if side == 0 else 1.0
                for a, k in enumerate(others):
                    gi[k] = si[a]
                    pt[k] = xg[si[a]]
                self.xf[f, s] = pt
                self.wf[s] = np.prod([wg[si[a]] for a in range(d - 1)])
                for jj in itertools.product(range(n1), repeat=d):
                    jj = tuple(reversed(jj))
                    j = tensor_index(jj, n1)
                    vals = []
                    for k in range(d):
                        vals.append(Bn[side, jj[k]] if k == r else B[gi[k], jj[k]])
                    self.phif[f, s, j] = np.prod(vals)
                    for kd in range(d):
                        dv = []
                        for k in range(d):
                            if k == r:
                                dv.append((Dn if kd == k else Bn)[side, jj[k]])
                            else:
                                dv.append((Dd if kd == k else B)[gi[k], jj[k]])
                        self.dphif[f, kd, s, j] = np.prod(dv)
            for li in itertools.product(range(n1), repeat=d - 1):
                li = tuple(reversed(li))
                lam = tensor_index(li, n1) if d > 1 else 0
                jj = [0] * d
                jj[r] = 0 if side == 0 else p
                for a, k in enumerate(others):
                    jj[k] = li[a]
                self.fnode[f, lam] = tensor_index(jj, n1)
        # trace basis at face points (same table for every face, local frame)
        self.mu = np.zeros((self.Nfq, self.Nfp))
        for si in itertools.product(range(q1), repeat=d - 1):
            si = tuple(reversed(si))
            s = tensor_index(si, q1) if d > 1 else 0
            for li in itertools.product(range(n1), repeat=d - 1):
                li = tuple(reversed(li))
                lam = tensor_index(li, n1) if d > 1 else 0
                self.mu[s, lam] = np.prod([B[si[a], li[a]] for a in range(d - 1)])
