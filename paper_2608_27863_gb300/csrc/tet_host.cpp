// Host set-up of tetrahedral handles: reference tables (Lagrange bases through
// a Legendre-product Vandermonde matrix, collapsed Gauss-Jacobi rules), the
// skeleton with canonical face frames and face degrees, quadratic geometry at
// the quadrature points of curved elements, and the per-element layout of the
// condensed system.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>

#include "tet.h"

namespace hdg {
namespace tet {
namespace {

const double kV[4][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
const int kFace[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
const int kEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
const double kOut[4][3] = {{1, 1, 1}, {-1, 0, 0}, {0, -1, 0}, {0, 0, -1}};
const int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// P_n^{(a,b)}(x) by the three-term recurrence of the Jacobi polynomials.
double jacobi(int n, double a, double b, double x) {
    if (n == 0) return 1.0;
    double p0 = 1.0, p1 = 0.5 * ((a + b + 2.0) * x + (a - b));
    for (int k = 2; k <= n; ++k) {
        const double c = 2.0 * k + a + b;
        const double a1 = 2.0 * k * (k + a + b) * (c - 2.0);
        const double a2 = (c - 1.0) * (a * a - b * b);
        const double a3 = (c - 2.0) * (c - 1.0) * c;
        const double a4 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * c;
        const double p2 = ((a2 + a3 * x) * p1 - a4 * p0) / a1;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

// d/dx P_n^{(a,b)} = (n + a + b + 1) / 2 P_{n-1}^{(a+1,b+1)}
double jacobi_deriv(int n, double a, double b, double x) {
    return n == 0 ? 0.0 : 0.5 * (n + a + b + 1.0) * jacobi(n - 1, a + 1.0, b + 1.0, x);
}

// n-point Gauss-Jacobi rule for the weight (1 - x)^alpha on [-1, 1]: roots by
// Newton's method with deflation (starting from the Chebyshev-Gauss points,
// each averaged with the previous root), weights 2^(alpha+1) / ((1 - x^2) P_n'(x)^2).
void gauss_jacobi(int n, int alpha, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int k = 0; k < n; ++k) {
        double r = -std::cos((2.0 * k + 1.0) * M_PI / (2.0 * n));
        if (k > 0) r = 0.5 * (r + x[k - 1]);
        for (int it = 0; it < 200; ++it) {
            double s = 0.0;
            for (int j = 0; j < k; ++j) s += 1.0 / (r - x[j]);
            const double P = jacobi(n, alpha, 0.0, r), dP = jacobi_deriv(n, alpha, 0.0, r);
            const double dl = -P / (dP - s * P);
            r += dl;
            if (std::fabs(dl) < 1e-16) break;
        }
        x[k] = r;
    }
    std::sort(x.begin(), x.end());
    for (int k = 0; k < n; ++k) {
        const double dP = jacobi_deriv(n, alpha, 0.0, x[k]);
        w[k] = std::pow(2.0, alpha + 1) / ((1.0 - x[k] * x[k]) * dP * dP);
    }
}

// Legendre values P_0..P_n and derivatives at x.
void legendre(int n, double x, double* P, double* dP) {
    P[0] = 1.0;
    dP[0] = 0.0;
    if (n >= 1) { P[1] = x; dP[1] = 1.0; }
    for (int k = 1; k < n; ++k) {
        P[k + 1] = ((2.0 * k + 1.0) * x * P[k] - k * P[k - 1]) / (k + 1.0);
        dP[k + 1] = (k >= 1 ? dP[k - 1] : 0.0) + (2.0 * k + 1.0) * P[k];
    }
}

std::vector<std::array<int, 3>> tet_lattice(int p) {
    std::vector<std::array<int, 3>> out;
    for (int k = 0; k <= p; ++k)
        for (int j = 0; j <= p - k; ++j)
            for (int i = 0; i <= p - j - k; ++i) out.push_back({i, j, k});
    return out;
}

std::vector<std::array<int, 2>> tri_lattice(int p) {
    std::vector<std::array<int, 2>> out;
    for (int j = 0; j <= p; ++j)
        for (int i = 0; i <= p - j; ++i) out.push_back({i, j});
    return out;
}

// Legendre-product basis P_i(x) P_j(y) P_k(z), (i, j, k) over the lattice: spans P_p.
void tet_modal(int p, const double* x, double* psi, double* dpsi /* [3][Np] or null */) {
    double Px[8], Py[8], Pz[8], dx[8], dy[8], dz[8];
    legendre(p, x[0], Px, dx);
    legendre(p, x[1], Py, dy);
    legendre(p, x[2], Pz, dz);
    const auto lat = tet_lattice(p);
    const int Np = (int)lat.size();
    for (int m = 0; m < Np; ++m) {
        const int i = lat[m][0], j = lat[m][1], k = lat[m][2];
        psi[m] = Px[i] * Py[j] * Pz[k];
        if (dpsi) {
            dpsi[m] = dx[i] * Py[j] * Pz[k];
            dpsi[Np + m] = Px[i] * dy[j] * Pz[k];
            dpsi[2 * Np + m] = Px[i] * Py[j] * dz[k];
        }
    }
}

void tri_modal(int p, const double* x, double* psi) {
    double Pr[8], Ps[8], d[8];
    legendre(p, x[0], Pr, d);
    legendre(p, x[1], Ps, d);
    const auto lat = tri_lattice(p);
    for (size_t m = 0; m < lat.size(); ++m) psi[m] = Pr[lat[m][0]] * Ps[lat[m][1]];
}

// Inverse of an n x n row-major matrix by Gauss-Jordan elimination with partial pivoting.
bool invert(int n, std::vector<double> A, std::vector<double>& inv) {
    inv.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
        if (A[(size_t)piv * n + c] == 0.0) return false;
        if (piv != c)
            for (int k = 0; k < n; ++k) {
                std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
                std::swap(inv[(size_t)c * n + k], inv[(size_t)piv * n + k]);
            }
        const double d = 1.0 / A[(size_t)c * n + c];
        for (int k = 0; k < n; ++k) { A[(size_t)c * n + k] *= d; inv[(size_t)c * n + k] *= d; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
                inv[(size_t)r * n + k] -= f * inv[(size_t)c * n + k];
            }
        }
    }
    return true;
}

// Vandermonde inverse of the tet basis of degree p on its equispaced nodes.
std::vector<double> tet_vinv(int p) {
    const auto lat = tet_lattice(p);
    const int Np = (int)lat.size();
    std::vector<double> V((size_t)Np * Np), inv;
    for (int n = 0; n < Np; ++n) {
        const double x[3] = {-1.0 + 2.0 * lat[n][0] / p, -1.0 + 2.0 * lat[n][1] / p, -1.0 + 2.0 * lat[n][2] / p};
        tet_modal(p, x, &V[(size_t)n * Np], nullptr);
    }
    invert(Np, V, inv);
    return inv;
}

// Lagrange basis values (and reference gradients) of degree p at point x.
void tet_lagrange(int p, const std::vector<double>& Vinv, const double* x, double* phi, double* dphi) {
    const int Np = n_tet(p);
    double psi[NPMAX], dpsi[3 * NPMAX];
    tet_modal(p, x, psi, dphi ? dpsi : nullptr);
    for (int j = 0; j < Np; ++j) {
        double s = 0.0;
        for (int m = 0; m < Np; ++m) s += psi[m] * Vinv[(size_t)m * Np + j];
        phi[j] = s;
        if (dphi)
            for (int r = 0; r < 3; ++r) {
                double t = 0.0;
                for (int m = 0; m < Np; ++m) t += dpsi[r * Np + m] * Vinv[(size_t)m * Np + j];
                dphi[r * Np + j] = t;
            }
    }
}

// Quadratic (10-node) shape function derivatives at reference point xi: dN [10][3].
void p2_dshape(const double* xi, double dN[10][3]) {
    const double lam[4] = {-(1.0 + xi[0] + xi[1] + xi[2]) / 2.0, (1.0 + xi[0]) / 2.0, (1.0 + xi[1]) / 2.0,
                           (1.0 + xi[2]) / 2.0};
    const double dl[4][3] = {{-0.5, -0.5, -0.5}, {0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5}};
    for (int i = 0; i < 4; ++i)
        for (int r = 0; r < 3; ++r) dN[i][r] = (4.0 * lam[i] - 1.0) * dl[i][r];
    for (int c = 0; c < 6; ++c) {
        const int a = kEdge[c][0], b = kEdge[c][1];
        for (int r = 0; r < 3; ++r) dN[4 + c][r] = 4.0 * (lam[a] * dl[b][r] + lam[b] * dl[a][r]);
    }
}

// J[k][r] = d x_k / d xi_r, det and inverse Jinv[r][k] = d xi_r / d x_k.
double jac_inv(const double J[3][3], double Ji[3][3]) {
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    // inverse = adjugate / det (adj[r][k] = cofactor of J[k][r])
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    return det;
}

int64_t master_of(const int64_t* pmap, int64_t nv, int64_t v) {
    if (!pmap) return v;
    for (int64_t guard = 0; guard <= nv && pmap[v] != v; ++guard) v = pmap[v];
    return v;
}

}  // namespace

void code_vertices(int code, int L[3]) {
    const int f = code / 6, s = code % 6;
    for (int k = 0; k < 3; ++k) L[k] = kFace[f][kPerm[s][k]];
}

void build_vol(int p, VolTab& t) {
    t.p = p;
    t.Np = n_tet(p);
    const int n = p + 2;
    t.Nq = n * n * n;
    std::vector<double> a, wa, b, wb, c, wc;
    gauss_jacobi(n, 0, a, wa);
    gauss_jacobi(n, 1, b, wb);
    gauss_jacobi(n, 2, c, wc);
    t.xq.assign((size_t)t.Nq * 3, 0.0);
    t.wq.assign(t.Nq, 0.0);
    for (int kc = 0, g = 0; kc < n; ++kc)
        for (int kb = 0; kb < n; ++kb)
            for (int ka = 0; ka < n; ++ka, ++g) {
                t.xq[g * 3 + 0] = (1 + a[ka]) * (1 - b[kb]) * (1 - c[kc]) / 4 - 1;
                t.xq[g * 3 + 1] = (1 + b[kb]) * (1 - c[kc]) / 2 - 1;
                t.xq[g * 3 + 2] = c[kc];
                t.wq[g] = wa[ka] * wb[kb] * wc[kc] / 8.0;
            }
    const auto Vinv = tet_vinv(p);
    t.phi.assign((size_t)t.Nq * t.Np, 0.0);
    t.dphi.assign((size_t)3 * t.Nq * t.Np, 0.0);
    for (int g = 0; g < t.Nq; ++g) {
        double dph[3 * NPMAX];
        tet_lagrange(p, Vinv, &t.xq[g * 3], &t.phi[(size_t)g * t.Np], dph);
        for (int r = 0; r < 3; ++r)
            for (int j = 0; j < t.Np; ++j) t.dphi[((size_t)r * t.Nq + g) * t.Np + j] = dph[r * t.Np + j];
    }
}

void build_tri(int p, TriTab& t) {
    t.p = p;
    t.Nfp = n_tri(p);
    const int n = p + 2;
    t.Nfq = n * n;
    std::vector<double> a, wa, b, wb;
    gauss_jacobi(n, 0, a, wa);
    gauss_jacobi(n, 1, b, wb);
    t.xs.assign((size_t)t.Nfq * 2, 0.0);
    t.ws.assign(t.Nfq, 0.0);
    for (int kb = 0, s = 0; kb < n; ++kb)
        for (int ka = 0; ka < n; ++ka, ++s) {
            t.xs[s * 2 + 0] = (1 + a[ka]) * (1 - b[kb]) / 2 - 1;
            t.xs[s * 2 + 1] = b[kb];
            t.ws[s] = wa[ka] * wb[kb] / 2.0;
        }
    const auto lat = tri_lattice(p);
    const int N = t.Nfp;
    std::vector<double> V((size_t)N * N), inv;
    for (int m = 0; m < N; ++m) {
        const double x[2] = {-1.0 + 2.0 * lat[m][0] / p, -1.0 + 2.0 * lat[m][1] / p};
        tri_modal(p, x, &V[(size_t)m * N]);
    }
    invert(N, V, inv);
    t.mu.assign((size_t)t.Nfq * N, 0.0);
    for (int s = 0; s < t.Nfq; ++s) {
        double psi[NFPMAX];
        tri_modal(p, &t.xs[s * 2], psi);
        for (int l = 0; l < N; ++l) {
            double v = 0.0;
            for (int m = 0; m < N; ++m) v += psi[m] * inv[(size_t)m * N + l];
            t.mu[(size_t)s * N + l] = v;
        }
    }
}

void build_face(int p, int pF, int code, std::vector<double>& phif, double nu[3]) {
    TriTab T;
    build_tri(pF, T);
    int L[3];
    code_vertices(code, L);
    const auto Vinv = tet_vinv(p);
    const int Np = n_tet(p);
    phif.assign((size_t)T.Nfq * Np, 0.0);
    for (int s = 0; s < T.Nfq; ++s) {
        const double m1 = (1.0 + T.xs[s * 2]) / 2.0, m2 = (1.0 + T.xs[s * 2 + 1]) / 2.0, m0 = 1.0 - m1 - m2;
        double xi[3];
        for (int r = 0; r < 3; ++r) xi[r] = m0 * kV[L[0]][r] + m1 * kV[L[1]][r] + m2 * kV[L[2]][r];
        tet_lagrange(p, Vinv, xi, &phif[(size_t)s * Np], nullptr);
    }
    double t1[3], t2[3];
    for (int r = 0; r < 3; ++r) { t1[r] = 0.5 * (kV[L[1]][r] - kV[L[0]][r]); t2[r] = 0.5 * (kV[L[2]][r] - kV[L[0]][r]); }
    nu[0] = t1[1] * t2[2] - t1[2] * t2[1];
    nu[1] = t1[2] * t2[0] - t1[0] * t2[2];
    nu[2] = t1[0] * t2[1] - t1[1] * t2[0];
    const int f = code / 6;
    if (nu[0] * kOut[f][0] + nu[1] * kOut[f][1] + nu[2] * kOut[f][2] < 0)
        for (int r = 0; r < 3; ++r) nu[r] = -nu[r];
}

int create_host(hdg_ctx* h, const hdg_tet_mesh* mesh, std::string& err) {
    if (!mesh || !mesh->vert_xyz || !mesh->elem_vert || !mesh->elem_p || mesh->n_elem <= 0 || mesh->n_vert <= 0) {
        err = "incomplete tetrahedral mesh";
        return HDG_EINVAL;
    }
    Ctx* c = new Ctx();
    h->tet = c;
    const int64_t E = mesh->n_elem, NV = mesh->n_vert;
    c->E = E;
    c->elem_p.assign(mesh->elem_p, mesh->elem_p + E);
    int pmax = 0;
    for (int64_t e = 0; e < E; ++e) {
        if (c->elem_p[e] < 1 || c->elem_p[e] > PMAX) { err = "element degree outside 1..4"; return HDG_EUNSUPPORTED; }
        pmax = std::max(pmax, c->elem_p[e]);
    }
    // skeleton: faces by sorted master ids, canonical frames
    std::map<std::array<int64_t, 3>, int32_t> fmap;
    c->e2f.assign((size_t)E * 4, -1);
    c->frame.assign((size_t)E * 12, 0);
    std::vector<int32_t> codes((size_t)E * 4);
    for (int64_t e = 0; e < E; ++e) {
        int64_t mv[4];
        for (int v = 0; v < 4; ++v) {
            const int64_t id = mesh->elem_vert[e * 4 + v];
            if (id < 0 || id >= NV) { err = "vertex index out of range"; return HDG_EINVAL; }
            mv[v] = master_of(mesh->periodic_map, NV, id);
        }
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b)
                if (mv[a] == mv[b]) { err = "element with repeated master vertices"; return HDG_EINVAL; }
        for (int f = 0; f < 4; ++f) {
            int L[3] = {kFace[f][0], kFace[f][1], kFace[f][2]};
            std::sort(L, L + 3, [&](int x, int y) { return mv[x] < mv[y]; });
            std::array<int64_t, 3> key = {mv[L[0]], mv[L[1]], mv[L[2]]};
            int code = -1;
            for (int s = 0; s < 6; ++s)
                if (kFace[f][kPerm[s][0]] == L[0] && kFace[f][kPerm[s][1]] == L[1] && kFace[f][kPerm[s][2]] == L[2])
                    code = f * 6 + s;
            codes[e * 4 + f] = code;
            for (int k = 0; k < 3; ++k) c->frame[(e * 4 + f) * 3 + k] = L[k];
            auto it = fmap.find(key);
            if (it == fmap.end()) {
                const int32_t F = (int32_t)c->f2e.size() / 2;
                fmap.emplace(key, F);
                c->f2e.push_back((int32_t)e);
                c->f2e.push_back(-1);
                c->f2lf.push_back(f);
                c->f2lf.push_back(-1);
                c->e2f[e * 4 + f] = F;
            } else {
                const int32_t F = it->second;
                if (c->f2e[2 * F + 1] != -1) { err = "face shared by more than two elements"; return HDG_EINVAL; }
                if (c->f2e[2 * F] == (int32_t)e) { err = "element on both sides of a face"; return HDG_EINVAL; }
                c->f2e[2 * F + 1] = (int32_t)e;
                c->f2lf[2 * F + 1] = f;
                c->e2f[e * 4 + f] = F;
            }
        }
    }
    const int64_t F = (int64_t)c->f2e.size() / 2;
    c->F = F;
    // boundary tags
    c->tags.assign((size_t)E * 4, 0);
    for (int64_t e = 0; e < E; ++e)
        for (int f = 0; f < 4; ++f) {
            const int32_t Fi = c->e2f[e * 4 + f];
            const bool bnd = c->f2e[2 * Fi + 1] < 0;
            const int tg = mesh->bnd_tag ? mesh->bnd_tag[e * 4 + f] : 0;
            if (tg < 0 || tg > 4) { err = "unsupported boundary tag"; return HDG_EUNSUPPORTED; }
            if (bnd && tg == 0) { err = "boundary face without a tag"; return HDG_EINVAL; }
            if (!bnd && tg != 0) { err = "interior face with a boundary tag"; return HDG_EINVAL; }
            c->tags[e * 4 + f] = tg;
            c->has_tag[tg] = true;
        }
    // face degrees and trace offsets
    c->face_p.assign(F, 0);
    for (int64_t Fi = 0; Fi < F; ++Fi) {
        int q = c->elem_p[c->f2e[2 * Fi]];
        if (c->f2e[2 * Fi + 1] >= 0) q = std::max(q, c->elem_p[c->f2e[2 * Fi + 1]]);
        c->face_p[Fi] = q;
    }
    c->hoff.assign(F + 1, 0);
    for (int64_t Fi = 0; Fi < F; ++Fi) c->hoff[Fi + 1] = c->hoff[Fi] + (int64_t)M * n_tri(c->face_p[Fi]);
    c->n_trace = c->hoff[F];
    c->uoff.assign(E + 1, 0);
    for (int64_t e = 0; e < E; ++e) c->uoff[e + 1] = c->uoff[e] + (int64_t)M * n_tet(c->elem_p[e]);
    c->n_u = c->uoff[E];
    // block pattern: row F, the faces of its elements (ascending)
    c->rowptr.assign(F + 1, 0);
    for (int64_t Fi = 0; Fi < F; ++Fi) {
        std::vector<int32_t> cols;
        for (int s = 0; s < 2; ++s) {
            const int32_t e = c->f2e[2 * Fi + s];
            if (e < 0) continue;
            for (int g = 0; g < 4; ++g) cols.push_back(c->e2f[e * 4 + g]);
        }
        std::sort(cols.begin(), cols.end());
        cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
        c->col.insert(c->col.end(), cols.begin(), cols.end());
        c->rowptr[Fi + 1] = (int32_t)c->col.size();
    }
    c->nnzb = (int64_t)c->col.size();
    c->boff.assign(c->nnzb + 1, 0);
    c->cptr.assign(c->nnzb + 1, 0);
    for (int64_t Fi = 0; Fi < F; ++Fi)
        for (int32_t b = c->rowptr[Fi]; b < c->rowptr[Fi + 1]; ++b) {
            const int32_t G = c->col[b];
            c->boff[b + 1] = c->boff[b] + (c->hoff[Fi + 1] - c->hoff[Fi]) * (c->hoff[G + 1] - c->hoff[G]);
            int32_t es[2] = {c->f2e[2 * Fi], c->f2e[2 * Fi + 1]};
            int32_t fs[2] = {c->f2lf[2 * Fi], c->f2lf[2 * Fi + 1]};
            if (es[1] >= 0 && es[1] < es[0]) { std::swap(es[0], es[1]); std::swap(fs[0], fs[1]); }
            for (int s = 0; s < 2; ++s) {
                if (es[s] < 0) continue;
                for (int g = 0; g < 4; ++g)
                    if (c->e2f[es[s] * 4 + g] == G) {
                        c->centry.push_back(es[s]);
                        c->centry.push_back(fs[s]);
                        c->centry.push_back(g);
                    }
            }
            c->cptr[b + 1] = (int32_t)(c->centry.size() / 3);
        }
    c->n_vals = c->boff[c->nnzb];
    c->diagb.assign(F, -1);
    c->bjoff.assign(F + 1, 0);
    for (int64_t Fi = 0; Fi < F; ++Fi) {
        for (int32_t b = c->rowptr[Fi]; b < c->rowptr[Fi + 1]; ++b)
            if (c->col[b] == (int32_t)Fi) c->diagb[Fi] = b;
        const int64_t bs = c->hoff[Fi + 1] - c->hoff[Fi];
        c->bjoff[Fi + 1] = c->bjoff[Fi] + bs * bs;
    }
    // reference tables
    c->vtab.assign(PMAX + 1, -1);
    c->ttab.assign(PMAX + 1, -1);
    c->ftab.assign((size_t)(PMAX + 1) * (PMAX + 1) * NCODE, -1);
    std::vector<VolTab> vt(PMAX + 1);
    std::vector<TriTab> tt(PMAX + 1);
    for (int p = 1; p <= PMAX; ++p) {
        build_vol(p, vt[p]);
        c->vtab[p] = (int32_t)c->tab.size();
        c->tab.insert(c->tab.end(), vt[p].phi.begin(), vt[p].phi.end());
        c->tab.insert(c->tab.end(), vt[p].dphi.begin(), vt[p].dphi.end());
        c->tab.insert(c->tab.end(), vt[p].wq.begin(), vt[p].wq.end());
        build_tri(p, tt[p]);
        c->ttab[p] = (int32_t)c->tab.size();
        c->tab.insert(c->tab.end(), tt[p].mu.begin(), tt[p].mu.end());
        c->tab.insert(c->tab.end(), tt[p].ws.begin(), tt[p].ws.end());
    }
    std::vector<double> fnu((size_t)(PMAX + 1) * (PMAX + 1) * NCODE * 3, 0.0);
    for (int p = 1; p <= pmax; ++p)
        for (int q = p; q <= pmax; ++q)
            for (int code = 0; code < NCODE; ++code) {
                std::vector<double> phif;
                double nu[3];
                build_face(p, q, code, phif, nu);
                const size_t k = ((size_t)p * (PMAX + 1) + q) * NCODE + code;
                c->ftab[k] = (int32_t)c->tab.size();
                c->tab.insert(c->tab.end(), phif.begin(), phif.end());
                c->tab.insert(c->tab.end(), nu, nu + 3);
                for (int r = 0; r < 3; ++r) fnu[k * 3 + r] = nu[r];
            }
    // per-element geometry and layout
    c->el.resize(E);
    h->centroid.assign((size_t)E * 3, 0.0);
    int64_t moff = 0, roff = 0, koff = 0;
    for (int64_t e = 0; e < E; ++e) {
        TetElem& d = c->el[e];
        std::memset(&d, 0, sizeof(d));
        const int p = c->elem_p[e];
        d.p = p;
        d.Np = n_tet(p);
        d.Nq = (p + 2) * (p + 2) * (p + 2);
        d.NU = M * d.Np;
        int t = 0, sfq = 0, sfp = 0;
        for (int f = 0; f < 4; ++f) {
            const int32_t Fi = c->e2f[e * 4 + f];
            d.face[f] = Fi;
            d.hoff[f] = c->hoff[Fi];
            d.pf[f] = c->face_p[Fi];
            d.code[f] = codes[e * 4 + f];
            d.tag[f] = c->tags[e * 4 + f];
            d.nfp[f] = n_tri(d.pf[f]);
            d.nfq[f] = (d.pf[f] + 2) * (d.pf[f] + 2);
            d.toff[f] = t;
            d.soff[f] = sfq;
            t += M * d.nfp[f];
            sfq += d.nfq[f];
            sfp += d.nfp[f];
            d.ftab[f] = c->ftab[((size_t)p * (PMAX + 1) + d.pf[f]) * NCODE + d.code[f]];
            d.ttab[f] = c->ttab[d.pf[f]];
        }
        d.t = t;
        d.sfq = sfq;
        d.LD = (d.NU + t + 1 + 1) & ~1;
        d.vtab = c->vtab[p];
        d.uoff = c->uoff[e];
        d.moff = moff;
        moff += (int64_t)(d.NU + t) * d.LD;
        d.roff = roff;
        roff += 3LL * d.Np * d.Np + 3LL * d.Np * sfp + 3LL * M * d.Np;
        d.koff = koff;
        koff += t;
        // geometry: quadratic nodes (given, or the straight-sided midpoints)
        double X[10][3];
        for (int v = 0; v < 4; ++v)
            for (int k = 0; k < 3; ++k)
                X[v][k] = mesh->geo ? mesh->geo[(e * 10 + v) * 3 + k]
                                    : mesh->vert_xyz[mesh->elem_vert[e * 4 + v] * 3 + k];
        double hmax = 0.0;
        for (int v = 1; v < 4; ++v)
            for (int k = 0; k < 3; ++k) hmax = std::max(hmax, std::fabs(X[v][k] - X[0][k]));
        for (int k = 0; k < 3; ++k) h->centroid[e * 3 + k] = 0.25 * (X[0][k] + X[1][k] + X[2][k] + X[3][k]);
        bool curved = false;
        for (int ed = 0; ed < 6; ++ed)
            for (int k = 0; k < 3; ++k) {
                const double mid = 0.5 * (X[kEdge[ed][0]][k] + X[kEdge[ed][1]][k]);
                X[4 + ed][k] = mesh->geo ? mesh->geo[(e * 10 + 4 + ed) * 3 + k] : mid;
                if (std::fabs(X[4 + ed][k] - mid) > 1e-12 * hmax) curved = true;
            }
        d.curved = curved ? 1 : 0;
        if (!curved) {
            double J[3][3], Ji[3][3];
            for (int k = 0; k < 3; ++k)
                for (int r = 0; r < 3; ++r) J[k][r] = 0.5 * (X[r + 1][k] - X[0][k]);
            d.detJ = jac_inv(J, Ji);
            if (!(d.detJ > 0.0)) { err = "non-positive Jacobian (element orientation)"; return HDG_EINVAL; }
            for (int r = 0; r < 3; ++r)
                for (int k = 0; k < 3; ++k) d.Jinv[r * 3 + k] = Ji[r][k];
            d.hinv = 1.0 / std::cbrt(4.0 / 3.0 * d.detJ);
            continue;
        }
        c->n_curved += 1;
        auto jac_at = [&](const double* xi, double J[3][3]) {
            double dN[10][3];
            p2_dshape(xi, dN);
            for (int k = 0; k < 3; ++k)
                for (int r = 0; r < 3; ++r) {
                    double s = 0.0;
                    for (int n = 0; n < 10; ++n) s += dN[n][r] * X[n][k];
                    J[k][r] = s;
                }
        };
        d.goff = (int64_t)c->gvol.size();
        const VolTab& V = vt[p];
        double vol = 0.0;
        for (int g = 0; g < d.Nq; ++g) {
            double J[3][3], Ji[3][3];
            jac_at(&V.xq[g * 3], J);
            const double det = jac_inv(J, Ji);
            if (!(det > 0.0)) { err = "non-positive Jacobian at a quadrature point"; return HDG_EINVAL; }
            vol += V.wq[g] * det;
            c->gvol.push_back(V.wq[g] * det);
            for (int r = 0; r < 3; ++r)
                for (int k = 0; k < 3; ++k) c->gvol.push_back(Ji[r][k]);
        }
        d.hinv = 1.0 / std::cbrt(vol);
        d.gfoff = (int64_t)c->gface.size();
        for (int f = 0; f < 4; ++f) {
            const TriTab& T = tt[d.pf[f]];
            int L[3];
            code_vertices(d.code[f], L);
            const double* nu = &fnu[(((size_t)p * (PMAX + 1) + d.pf[f]) * NCODE + d.code[f]) * 3];
            for (int s = 0; s < T.Nfq; ++s) {
                const double m1 = (1.0 + T.xs[s * 2]) / 2.0, m2 = (1.0 + T.xs[s * 2 + 1]) / 2.0, m0 = 1.0 - m1 - m2;
                double xi[3], J[3][3], Ji[3][3];
                for (int r = 0; r < 3; ++r) xi[r] = m0 * kV[L[0]][r] + m1 * kV[L[1]][r] + m2 * kV[L[2]][r];
                jac_at(xi, J);
                const double det = jac_inv(J, Ji);
                if (!(det > 0.0)) { err = "non-positive Jacobian at a face point"; return HDG_EINVAL; }
                for (int k = 0; k < 3; ++k) {
                    double s2 = 0.0;
                    for (int r = 0; r < 3; ++r) s2 += Ji[r][k] * nu[r];
                    c->gface.push_back(T.ws[s] * det * s2);
                }
            }
        }
    }
    c->n_mat = moff;
    c->n_rec = roff;
    c->n_rk = koff;
    // persistent launch order: decreasing estimated FP64 work, ties by element id
    std::vector<double> cost(E);
    for (int64_t e = 0; e < E; ++e) {
        const TetElem& d = c->el[e];
        const double nu = d.NU, t = d.t, nc = d.Np + d.t / M;
        cost[e] = 50.0 * d.Np * nc * (3.0 * d.Nq + d.sfq) + nu * nu * nu + 2.0 * nu * (nu + t) * (t + 1);
    }
    c->order.resize(E);
    for (int64_t e = 0; e < E; ++e) c->order[e] = (int32_t)e;
    std::stable_sort(c->order.begin(), c->order.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
    // handle-level fields read by shared entry points
    h->d = 3;
    h->m = M;
    h->p = pmax;
    h->E = E;
    h->F = F;
    h->nnzb = c->nnzb;
    h->has_bnd = false;
    for (int k = 1; k <= 4; ++k) {
        h->has_tag[k] = c->has_tag[k];
        h->has_bnd = h->has_bnd || c->has_tag[k];
    }
    return HDG_OK;
}

}  // namespace tet
}  // namespace hdg

extern "C" {

int hdg_tet_ref_tables(int p, double* xq, double* wq, double* phi, double* dphi) {
    if (p < 1 || p > hdg::tet::PMAX) return HDG_EUNSUPPORTED;
    hdg::tet::VolTab t;
    hdg::tet::build_vol(p, t);
    if (xq) std::memcpy(xq, t.xq.data(), t.xq.size() * sizeof(double));
    if (wq) std::memcpy(wq, t.wq.data(), t.wq.size() * sizeof(double));
    if (phi) std::memcpy(phi, t.phi.data(), t.phi.size() * sizeof(double));
    if (dphi) std::memcpy(dphi, t.dphi.data(), t.dphi.size() * sizeof(double));
    return HDG_OK;
}

int hdg_tri_ref_tables(int pF, double* xs, double* ws, double* mu) {
    if (pF < 1 || pF > hdg::tet::PMAX) return HDG_EUNSUPPORTED;
    hdg::tet::TriTab t;
    hdg::tet::build_tri(pF, t);
    if (xs) std::memcpy(xs, t.xs.data(), t.xs.size() * sizeof(double));
    if (ws) std::memcpy(ws, t.ws.data(), t.ws.size() * sizeof(double));
    if (mu) std::memcpy(mu, t.mu.data(), t.mu.size() * sizeof(double));
    return HDG_OK;
}

}  // extern "C"
