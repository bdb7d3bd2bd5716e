// Skeleton connectivity of the HDG trace space (host).
//
// Faces are identified through their master vertices (periodic faces are
// paired, Sec. 2.1 boundary paragraph) and numbered by first encounter over
// (element, local face).  Trace nodes of a face are ordered in a canonical
// frame independent of the element that sees it: origin at the corner with
// the smallest master id, first axis towards the adjacent corner with the
// smaller id.  Each element stores the map from its local face-node order to
// the canonical one as the affine index map
//     local = p * O + k1 * (A1 - O) + k2 * (A2 - O)
// in the face's corner coordinates (O origin, A1 / A2 the axis corners).
// The block-sparse trace matrix has one block row per face and a block for
// every face sharing an element with it (Sec. 3.2, 3.5), columns ascending.
#include <algorithm>
#include <array>
#include <map>

#include "common.h"

namespace hdg {
namespace {

int64_t master_of(const hdg_mesh& m, int64_t v, bool& ok) {
    if (!m.periodic_map) return v;
    for (int it = 0; it < 64; ++it) {
        int64_t w = m.periodic_map[v];
        if (w < 0 || w >= m.n_vert) { ok = false; return v; }
        if (w == v) return v;
        v = w;
    }
    ok = false;  // cycle
    return v;
}

// element vertex numbers of local face f in the face's local corner order
void face_corner_vertices(int d, int f, int* out) {
    int r = f / 2, side = f % 2;
    int nc = 1 << (d - 1);
    for (int c = 0; c < nc; ++c) {
        int v = side << r, a = 0;
        for (int k = 0; k < d; ++k) {
            if (k == r) continue;
            v |= ((c >> a) & 1) << k;
            ++a;
        }
        out[c] = v;
    }
}

}  // namespace

int build_skeleton(const hdg_mesh& mesh, int p, Skeleton& s, std::string& err) {
    const int d = mesh.dim, nf = 2 * d, n1 = p + 1;
    const int Nfp = ipow(n1, d - 1), nc = 1 << (d - 1);
    const int64_t E = mesh.n_elem;
    std::map<std::array<int64_t, 4>, int32_t> key2face;
    s.e2f.assign((size_t)E * nf, -1);
    s.f2e.clear(); s.f2lf.clear();
    std::vector<std::array<int64_t, 4>> corner_ids;  // per element-face, local corner order
    corner_ids.resize((size_t)E * nf);
    bool ok = true;
    for (int64_t e = 0; e < E; ++e) {
        for (int f = 0; f < nf; ++f) {
            int cv[4];
            face_corner_vertices(d, f, cv);
            std::array<int64_t, 4> ids{-1, -1, -1, -1};
            for (int c = 0; c < nc; ++c) {
                int64_t v = mesh.elem_vert[(size_t)e * (1 << d) + cv[c]];
                if (v < 0 || v >= mesh.n_vert) { err = "elem_vert out of range"; return HDG_EINVAL; }
                ids[c] = master_of(mesh, v, ok);
            }
            if (!ok) { err = "periodic_map out of range or cyclic"; return HDG_EINVAL; }
            corner_ids[(size_t)e * nf + f] = ids;
            std::array<int64_t, 4> key = ids;
            std::sort(key.begin(), key.begin() + nc);
            for (int c = 1; c < nc; ++c)
                if (key[c] == key[c - 1]) { err = "degenerate face (periodic direction with fewer than 2 elements?)"; return HDG_EINVAL; }
            auto it = key2face.find(key);
            if (it == key2face.end()) {
                int32_t F = (int32_t)(s.f2e.size() / 2);
                key2face.emplace(key, F);
                s.f2e.push_back((int32_t)e); s.f2e.push_back(-1);
                s.f2lf.push_back(f); s.f2lf.push_back(-1);
                s.e2f[(size_t)e * nf + f] = F;
            } else {
                int32_t F = it->second;
                if (s.f2e[2 * F + 1] != -1) { err = "a face is shared by more than two elements"; return HDG_EINVAL; }
                if (s.f2e[2 * F] == (int32_t)e) { err = "an element lies on both sides of a face (periodic direction too short)"; return HDG_EINVAL; }
                s.f2e[2 * F + 1] = (int32_t)e; s.f2lf[2 * F + 1] = f;
                s.e2f[(size_t)e * nf + f] = F;
            }
        }
    }
    s.n_faces = (int64_t)s.f2e.size() / 2;

    // orientation maps
    s.perm.assign((size_t)E * nf * Nfp, 0);
    s.iperm.assign((size_t)E * nf * Nfp, 0);
    for (int64_t e = 0; e < E; ++e)
        for (int f = 0; f < nf; ++f) {
            const std::array<int64_t, 4>& ids = corner_ids[(size_t)e * nf + f];
            int O = 0;
            for (int c = 1; c < nc; ++c) if (ids[c] < ids[O]) O = c;
            int32_t* pm = &s.perm[((size_t)e * nf + f) * Nfp];
            int32_t* ipm = &s.iperm[((size_t)e * nf + f) * Nfp];
            if (d == 2) {
                int A = O ^ 1;
                int step = (A & 1) - (O & 1);            // +1 or -1
                for (int k = 0; k < n1; ++k) {
                    int loc = p * (O & 1) + k * step;
                    pm[loc] = k; ipm[k] = loc;
                }
            } else {
                int N0 = O ^ 1, N1 = O ^ 2;
                int A1 = ids[N0] < ids[N1] ? N0 : N1;
                int A2 = (A1 == N0) ? N1 : N0;
                int o[2] = {O & 1, (O >> 1) & 1};
                int e1[2] = {(A1 & 1) - o[0], ((A1 >> 1) & 1) - o[1]};
                int e2[2] = {(A2 & 1) - o[0], ((A2 >> 1) & 1) - o[1]};
                for (int k2 = 0; k2 < n1; ++k2)
                    for (int k1 = 0; k1 < n1; ++k1) {
                        int l0 = p * o[0] + k1 * e1[0] + k2 * e2[0];
                        int l1 = p * o[1] + k1 * e1[1] + k2 * e2[1];
                        int loc = l0 + n1 * l1, can = k1 + n1 * k2;
                        pm[loc] = can; ipm[can] = loc;
                    }
            }
        }

    // block pattern
    const int64_t F = s.n_faces;
    s.rowptr.assign(F + 1, 0);
    std::vector<std::vector<int32_t>> rows(F);
    for (int64_t f = 0; f < F; ++f) {
        std::vector<int32_t>& r = rows[f];
        for (int side = 0; side < 2; ++side) {
            int32_t e = s.f2e[2 * f + side];
            if (e < 0) continue;
            for (int k = 0; k < nf; ++k) r.push_back(s.e2f[(size_t)e * nf + k]);
        }
        std::sort(r.begin(), r.end());
        r.erase(std::unique(r.begin(), r.end()), r.end());
        s.rowptr[f + 1] = s.rowptr[f] + (int32_t)r.size();
    }
    s.col.resize(s.rowptr[F]);
    for (int64_t f = 0; f < F; ++f) std::copy(rows[f].begin(), rows[f].end(), s.col.begin() + s.rowptr[f]);

    // per element: block of each (fl, gl) pair and the rank of its contribution
    s.blk.assign((size_t)E * nf * nf, 0);
    s.rank.assign((size_t)E * nf * nf, 0);
    s.frank.assign((size_t)E * nf, 0);
    for (int64_t e = 0; e < E; ++e)
        for (int fl = 0; fl < nf; ++fl) {
            int32_t Fi = s.e2f[(size_t)e * nf + fl];
            s.frank[(size_t)e * nf + fl] = (s.f2e[2 * Fi] == (int32_t)e) ? 0 : 1;
            for (int gl = 0; gl < nf; ++gl) {
                int32_t G = s.e2f[(size_t)e * nf + gl];
                const int32_t* b0 = &s.col[s.rowptr[Fi]];
                const int32_t* b1 = &s.col[s.rowptr[Fi + 1]];
                const int32_t* it = std::lower_bound(b0, b1, G);
                s.blk[((size_t)e * nf + fl) * nf + gl] = (int32_t)(it - &s.col[0]);
                int rk = 0;
                for (int side = 0; side < 2; ++side) {
                    int32_t e2 = s.f2e[2 * Fi + side];
                    if (e2 < 0 || e2 >= (int32_t)e) continue;
                    for (int k = 0; k < nf; ++k)
                        if (s.e2f[(size_t)e2 * nf + k] == G) { ++rk; break; }
                }
                s.rank[((size_t)e * nf + fl) * nf + gl] = rk;
            }
        }
    return HDG_OK;
}

// Master vertices of every element corner, renumbered compactly in order of
// first appearance, and the vertex -> element lists (ascending element ids):
// the vertex averaging of the artificial-viscosity smoothing.
int build_vertex_map(const hdg_mesh& mesh, std::vector<int32_t>& ev, std::vector<int32_t>& vrow,
                     std::vector<int32_t>& vcol, std::string& err) {
    const int nv = 1 << mesh.dim;
    const int64_t E = mesh.n_elem;
    std::vector<int32_t> id((size_t)mesh.n_vert, -1);
    ev.assign((size_t)E * nv, 0);
    int32_t nmaster = 0;
    for (int64_t e = 0; e < E; ++e)
        for (int c = 0; c < nv; ++c) {
            bool ok = true;
            const int64_t v = master_of(mesh, mesh.elem_vert[(size_t)e * nv + c], ok);
            if (!ok) { err = "periodic_map out of range or cyclic"; return HDG_EINVAL; }
            if (id[v] < 0) id[v] = nmaster++;
            ev[(size_t)e * nv + c] = id[v];
        }
    vrow.assign((size_t)nmaster + 1, 0);
    for (int64_t i = 0; i < E * nv; ++i) ++vrow[ev[i] + 1];
    for (int32_t v = 0; v < nmaster; ++v) vrow[v + 1] += vrow[v];
    vcol.assign((size_t)E * nv, 0);
    std::vector<int32_t> fill(vrow.begin(), vrow.end() - 1);
    for (int64_t e = 0; e < E; ++e)
        for (int c = 0; c < nv; ++c) vcol[fill[ev[(size_t)e * nv + c]]++] = (int32_t)e;
    return HDG_OK;
}

}  // namespace hdg
