// Partition-ready layout of a mesh for a run over several GPUs (Sec. 3.5):
// element-local work (linearization, condensation, recovery) stays on the part
// that owns the element, and the parts exchange only trace data of faces on
// part interfaces: condensed face blocks during assembly and trace entries in
// every matvec.  Host only; nothing here communicates.
#include <algorithm>
#include <cmath>
#include <limits>
#include <numeric>
#include <string>
#include <vector>

#include "common.h"
#include "tet.h"

namespace {

// face-element adjacency and block pattern, for either kind of handle
struct MeshView {
    int64_t E = 0, F = 0;
    const int32_t* f2e = nullptr;       // [F][2] element ids, -1 for the missing side of a boundary face
    const int32_t* rowptr = nullptr;    // [F + 1] block rows
    const int32_t* col = nullptr;
    const double* centroid = nullptr;   // [E][3]
};

MeshView mesh_view(hdg_ctx* h) {
    MeshView v;
    if (h->tet) {
        const hdg::tet::Ctx* c = h->tet;
        v.E = c->E; v.F = c->F;
        v.f2e = c->f2e.data(); v.rowptr = c->rowptr.data(); v.col = c->col.data();
    } else {
        v.E = h->E; v.F = h->sk.n_faces;
        v.f2e = h->sk.f2e.data(); v.rowptr = h->sk.rowptr.data(); v.col = h->sk.col.data();
    }
    v.centroid = h->centroid.data();
    return v;
}

int fail_h(hdg_ctx* h, int code, const std::string& msg) {
    h->err = msg;
    return code;
}

// elements of part q when E elements go to P parts: the first E mod P parts take one more
int64_t part_size(int64_t E, int P, int q) { return E / P + (q < E % P ? 1 : 0); }

// Recursive coordinate bisection: ids[lo, hi) go to parts [q0, q0 + np).  The set is
// split across the longest extent of its centroids (lowest axis on ties) at the
// number of elements of the first np / 2 parts, ordered by (coordinate, element id).
void rcb(const double* cen, std::vector<int64_t>& ids, int64_t lo, int64_t hi, int q0, int np, int64_t E, int P,
         int32_t* part) {
    if (np == 1) {
        for (int64_t i = lo; i < hi; ++i) part[ids[i]] = q0;
        return;
    }
    double mn[3], mx[3];
    for (int k = 0; k < 3; ++k) {
        mn[k] = std::numeric_limits<double>::infinity();
        mx[k] = -std::numeric_limits<double>::infinity();
    }
    for (int64_t i = lo; i < hi; ++i)
        for (int k = 0; k < 3; ++k) {
            mn[k] = std::min(mn[k], cen[ids[i] * 3 + k]);
            mx[k] = std::max(mx[k], cen[ids[i] * 3 + k]);
        }
    int ax = 0;
    for (int k = 1; k < 3; ++k)
        if (mx[k] - mn[k] > mx[ax] - mn[ax]) ax = k;
    const int n1 = np / 2;
    int64_t c1 = 0;
    for (int q = q0; q < q0 + n1; ++q) c1 += part_size(E, P, q);
    auto before = [&](int64_t a, int64_t b) {
        const double xa = cen[a * 3 + ax], xb = cen[b * 3 + ax];
        return xa < xb || (xa == xb && a < b);
    };
    std::nth_element(ids.begin() + lo, ids.begin() + lo + c1, ids.begin() + hi, before);
    rcb(cen, ids, lo, lo + c1, q0, n1, E, P, part);
    rcb(cen, ids, lo + c1, hi, q0 + n1, np - n1, E, P, part);
}

}  // namespace

extern "C" {

int hdg_partition(hdg_handle h, int n_parts, int32_t* elem_part) {
    if (!h) return HDG_EINVAL;
    if (!elem_part) return fail_h(h, HDG_EINVAL, "elem_part is required");
    const MeshView v = mesh_view(h);
    if (n_parts < 1 || n_parts > v.E) return fail_h(h, HDG_EINVAL, "n_parts must be in 1..n_elem");
    if ((int64_t)h->centroid.size() != 3 * v.E) return fail_h(h, HDG_EINVAL, "handle has no element centroids");
    std::vector<int64_t> ids(v.E);
    std::iota(ids.begin(), ids.end(), 0);
    rcb(v.centroid, ids, 0, v.E, 0, n_parts, v.E, n_parts, elem_part);
    return HDG_OK;
}

int hdg_part_layout(hdg_handle h, const int32_t* elem_part, int part, hdg_part_sizes* sizes, int64_t* elems,
                    int64_t* faces, int64_t* interface_faces, int32_t* interface_peer, int64_t* halo_faces,
                    int32_t* halo_owner) {
    if (!h) return HDG_EINVAL;
    if (!elem_part || part < 0) return fail_h(h, HDG_EINVAL, "elem_part and part >= 0 are required");
    const MeshView v = mesh_view(h);
    for (int64_t e = 0; e < v.E; ++e)
        if (elem_part[e] < 0) return fail_h(h, HDG_EINVAL, "negative part id at element " + std::to_string(e));
    // owner of a face: the smaller part id of its elements
    std::vector<int32_t> owner(v.F);
    std::vector<char> on_interface(v.E, 0);
    hdg_part_sizes s{};
    for (int64_t F = 0; F < v.F; ++F) {
        const int32_t e0 = v.f2e[2 * F], e1 = v.f2e[2 * F + 1];
        const int32_t p0 = e0 >= 0 ? elem_part[e0] : elem_part[e1];
        const int32_t p1 = e1 >= 0 ? elem_part[e1] : p0;
        owner[F] = std::min(p0, p1);
        if (p0 != p1) {
            on_interface[e0] = on_interface[e1] = 1;
            if (p0 == part || p1 == part) {
                if (interface_faces) interface_faces[s.n_interface_faces] = F;
                if (interface_peer) interface_peer[s.n_interface_faces] = p0 == part ? p1 : p0;
                ++s.n_interface_faces;
            }
        }
        if (owner[F] == part) {
            if (faces) faces[s.n_faces] = F;
            ++s.n_faces;
        }
    }
    for (int pass = 0; pass < 2; ++pass)                      // interior elements, then interface elements
        for (int64_t e = 0; e < v.E; ++e)
            if (elem_part[e] == part && on_interface[e] == pass) {
                if (elems) elems[s.n_elem] = e;
                ++s.n_elem;
                if (pass == 0) ++s.n_interior_elem;
            }
    // halo: faces owned elsewhere that the owned block rows reference
    std::vector<int64_t> halo;
    for (int64_t F = 0; F < v.F; ++F) {
        if (owner[F] != part) continue;
        for (int32_t b = v.rowptr[F]; b < v.rowptr[F + 1]; ++b)
            if (owner[v.col[b]] != part) halo.push_back(v.col[b]);
    }
    std::sort(halo.begin(), halo.end());
    halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
    s.n_halo_faces = (int64_t)halo.size();
    for (size_t i = 0; i < halo.size(); ++i) {
        if (halo_faces) halo_faces[i] = halo[i];
        if (halo_owner) halo_owner[i] = owner[halo[i]];
    }
    if (sizes) *sizes = s;
    return HDG_OK;
}

}  // extern "C"
