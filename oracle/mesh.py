"""Skeleton connectivity: faces, orientation permutations, block-sparse pattern.

Oracle (test infrastructure only).  The mesh skeleton of Sec. 2.2 and the
face-partitioned trace vector of Sec. 3.5, with these readings (the paper does
not fix an ordering):

* vertices are first replaced by their periodic master (periodic faces are
  identified, Sec. 2.1 boundary paragraph);
* faces are numbered in order of first encounter scanning elements
  ``e = 0..E-1`` and local faces ``f = 0..2d-1``;
* a face's canonical node frame has its origin at the corner with the smallest
  master vertex id; the first axis points to the adjacent corner with the
  smaller id, the second to the other; canonical node ``k1 + (p+1) k2``;
* the block-sparse trace matrix has one block row per face, with a block for
  every face sharing an element with it, columns ascending;
* a block's contributions are summed in ascending element order.
"""
from __future__ import annotations

import numpy as np


def face_corners(d: int, f: int):
    """Element vertex numbers of local face f, in the face's local order."""
    r, side = divmod(f, 2)
    others = [k for k in range(d) if k != r]
    out = []
    for c in range(2 ** (d - 1)):
        v = side << r
        for a, k in enumerate(others):
            v |= ((c >> a) & 1) << k
        out.append(v)
    return out


def master(pmap: np.ndarray, v: int) -> int:
    while pmap[v] != v:
        v = int(pmap[v])
    return int(v)


class Connectivity:
    """Face numbering, element-to-face maps, permutations and the BSR pattern.

    * ``f2e[F] = [(e0, f0), (e1, f1)]`` (second entry ``(-1, -1)`` on the boundary);
    * ``e2f[e, f]`` global face of local face f;
    * ``perm[e, f, l]`` canonical index of local face node l;
    * ``rowptr``, ``col`` block pattern; ``contrib[b]`` list of ``(e, fl, gl)``.
    """

    def __init__(self, mesh, p: int):
        d = mesh.dim
        nf = 2 * d
        n1 = p + 1
        Nfp = n1 ** (d - 1)
        E = mesh.n_elem
        pmap = np.asarray(mesh.periodic_map)
        ev = np.asarray(mesh.elem_vert)
        key2face = {}
        f2e = []
        self.e2f = np.zeros((E, nf), dtype=np.int64)
        self.corner_ids = []
        for e in range(E):
            for f in range(nf):
                ids = [master(pmap, int(ev[e, c])) for c in face_corners(d, f)]
                key = tuple(sorted(ids))
                if len(set(ids)) != len(ids):
                    raise ValueError("degenerate face (periodic direction too short)")
                if key not in key2face:
                    key2face[key] = len(f2e)
                    f2e.append([(e, f), (-1, -1)])
                    self.corner_ids.append(ids)
                else:
                    F = key2face[key]
                    if f2e[F][1] != (-1, -1):
                        raise ValueError("face shared by more than two elements")
                    f2e[F][1] = (e, f)
                self.e2f[e, f] = key2face[key]
        self.n_faces = len(f2e)
        self.f2e = np.array(f2e, dtype=np.int64)  # [F][2][2]

        # orientation permutations
        self.perm = np.zeros((E, nf, Nfp), dtype=np.int64)
        for e in range(E):
            for f in range(nf):
                ids = [master(pmap, int(ev[e, c])) for c in face_corners(d, f)]
                self.perm[e, f] = self._perm(ids, d, p)

        # block pattern
        rows = []
        for F in range(self.n_faces):
            nb = set()
            for (e, f) in self.f2e[F]:
                if e >= 0:
                    nb.update(int(x) for x in self.e2f[e])
            rows.append(sorted(nb))
        self.rowptr = np.zeros(self.n_faces + 1, dtype=np.int64)
        for F in range(self.n_faces):
            self.rowptr[F + 1] = self.rowptr[F] + len(rows[F])
        self.col = np.array([c for r in rows for c in r], dtype=np.int64)
        self.contrib = []
        for F in range(self.n_faces):
            for b in range(self.rowptr[F], self.rowptr[F + 1]):
                G = int(self.col[b])
                lst = []
                for (e, _) in self.f2e[F]:  # the elements of F, ascending
                    if e < 0:
                        continue
                    fs = [int(x) for x in self.e2f[e]]
                    if G in fs:
                        lst.append((int(e), fs.index(F), fs.index(G)))
                self.contrib.append(sorted(lst))

    @staticmethod
    def _perm(ids, d, p):
        """Local face node -> canonical face node (reading of the frame above)."""
        n1 = p + 1
        if d == 2:
            o = 0 if ids[0] < ids[1] else 1
            return np.array([l if o == 0 else p - l for l in range(n1)], dtype=np.int64)
        o = int(np.argmin(ids))
        nbrs = [o ^ 1, o ^ 2]  # corners differing in local direction 0 / 1
        if ids[nbrs[0]] < ids[nbrs[1]]:
            dir1, dir2 = 0, 1
        else:
            dir1, dir2 = 1, 0
        out = np.zeros(n1 * n1, dtype=np.int64)
        obits = [(o >> 0) & 1, (o >> 1) & 1]
        for k2 in range(n1):
            for k1 in range(n1):
                loc = [0, 0]
                loc[dir1] = k1 if obits[dir1] == 0 else p - k1
                loc[dir2] = k2 if obits[dir2] == 0 else p - k2
                out[loc[0] + n1 * loc[1]] = k1 + n1 * k2
        return out

    def block_index(self, F: int, G: int) -> int:
        lo, hi = self.rowptr[F], self.rowptr[F + 1]
        for b in range(lo, hi):
            if self.col[b] == G:
                return int(b)
        raise KeyError((F, G))
