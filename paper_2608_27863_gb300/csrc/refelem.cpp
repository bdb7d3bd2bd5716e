// Reference-element tables for tensor-product HDG elements (host, FP64).
//
// Spaces of Sec. 2.2 (eq. spaces) taken as the tensor space Q^k on [-1, 1]^d:
// nodal Lagrange bases on Gauss-Lobatto points, Gauss-Legendre quadrature with
// p + 2 points per direction, trace bases on each face's own Gauss-Lobatto
// points.  Besides the plain tables this file precomputes the operators used to
// eliminate the gradient unknowns exactly: with the reference mass matrix
// Mhat, Chat_r[i][j] = (d_r phi_i, phi_j) and Ehat_f[i][l] = <phi_i, mu_l>_f,
// it stores Mhat^{-1} Chat_r, Mhat^{-1} Ehat_f and their values at the volume
// and face quadrature points.
#include <cmath>
#include <stdexcept>

#include "common.h"

namespace hdg {
namespace {

// Legendre P_n(x) and P_n'(x) by the three-term recurrence.
void legendre(int n, double x, double& P, double& dP) {
    double p0 = 1.0, p1 = x;
    if (n == 0) { P = 1.0; dP = 0.0; return; }
    for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1; p1 = p2;
    }
    P = p1;
    dP = n * (x * p1 - p0) / (x * x - 1.0);
}

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0); w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = -std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            legendre(n, z, P, dP);
            double dz = P / dP;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double P, dP;
        legendre(n, z, P, dP);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dP * dP);
    }
}

// Gauss-Lobatto nodes of degree p: +-1 and the roots of P_p', found by Newton
// with P_p'' from Legendre's equation.
std::vector<double> gll(int p) {
    std::vector<double> x(p + 1);
    x[0] = -1.0; x[p] = 1.0;
    for (int i = 1; i < p; ++i) {
        double z = -std::cos(M_PI * i / p);
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            legendre(p, z, P, dP);
            double d2P = (2.0 * z * dP - p * (p + 1.0) * P) / (1.0 - z * z);
            double dz = dP / d2P;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
    }
    return x;
}

// Barycentric Lagrange interpolation: values and derivatives at point x.
struct Lagrange1D {
    std::vector<double> xn, bw;
    explicit Lagrange1D(const std::vector<double>& nodes) : xn(nodes), bw(nodes.size(), 1.0) {
        int n = (int)xn.size();
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k)
                if (k != j) bw[j] /= (xn[j] - xn[k]);
    }
    void eval(double x, double* val, double* der) const {
        int n = (int)xn.size();
        int hit = -1;
        for (int j = 0; j < n; ++j)
            if (x == xn[j]) hit = j;
        if (hit >= 0) {
            // at a node: cardinal values; derivative row of the differentiation matrix
            for (int j = 0; j < n; ++j) val[j] = (j == hit) ? 1.0 : 0.0;
            double diag = 0.0;
            for (int j = 0; j < n; ++j) {
                if (j == hit) continue;
                der[j] = (bw[j] / bw[hit]) / (xn[hit] - xn[j]);
                diag -= der[j];
            }
            der[hit] = diag;
            return;
        }
        double s = 0.0, sd = 0.0;
        std::vector<double> t(n);
        for (int j = 0; j < n; ++j) { t[j] = bw[j] / (x - xn[j]); s += t[j]; }
        for (int j = 0; j < n; ++j) val[j] = t[j] / s;
        // l_j'(x) = l_j(x) * (sum_k 1/(x - x_k) - 1/(x - x_j)) computed stably:
        for (int j = 0; j < n; ++j) sd += t[j] / (x - xn[j]);
        for (int j = 0; j < n; ++j) der[j] = val[j] * (sd / s - 1.0 / (x - xn[j]));
    }
};

void invert(std::vector<double> a, int n, std::vector<double>& inv) {
    inv.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(a[(size_t)r * n + c]) > std::fabs(a[(size_t)piv * n + c])) piv = r;
        if (a[(size_t)piv * n + c] == 0.0) throw std::runtime_error("singular reference mass matrix");
        for (int k = 0; k < n; ++k) {
            std::swap(a[(size_t)c * n + k], a[(size_t)piv * n + k]);
            std::swap(inv[(size_t)c * n + k], inv[(size_t)piv * n + k]);
        }
        double s = 1.0 / a[(size_t)c * n + c];
        for (int k = 0; k < n; ++k) { a[(size_t)c * n + k] *= s; inv[(size_t)c * n + k] *= s; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double f = a[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                a[(size_t)r * n + k] -= f * a[(size_t)c * n + k];
                inv[(size_t)r * n + k] -= f * inv[(size_t)c * n + k];
            }
        }
    }
}

}  // namespace

void build_ref_tables(int d, int p, RefTables& t) {
    t.d = d; t.p = p;
    const int n1 = p + 1, q1 = p + 2;
    t.Np = ipow(n1, d); t.Nq = ipow(q1, d);
    t.nf = 2 * d; t.Nfp = ipow(n1, d - 1); t.Nfq = ipow(q1, d - 1);
    const int Np = t.Np, Nq = t.Nq, nf = t.nf, Nfp = t.Nfp, Nfq = t.Nfq;
    t.nodes1 = gll(p);
    gauss_legendre(q1, t.gq1, t.gw1);
    Lagrange1D L(t.nodes1);
    // 1-D tables at Gauss points and at the end points
    std::vector<double> B((size_t)q1 * n1), Dd((size_t)q1 * n1), Be(2 * n1), De(2 * n1);
    for (int g = 0; g < q1; ++g) L.eval(t.gq1[g], &B[(size_t)g * n1], &Dd[(size_t)g * n1]);
    L.eval(-1.0, &Be[0], &De[0]);
    L.eval(1.0, &Be[n1], &De[n1]);
    t.b1 = B;
    t.d1 = Dd;

    auto digit = [](int idx, int base, int r) { for (int k = 0; k < r; ++k) idx /= base; return idx % base; };

    t.phi.assign((size_t)Nq * Np, 0.0);
    t.dphi.assign((size_t)d * Nq * Np, 0.0);
    t.wq.assign(Nq, 0.0);
    for (int g = 0; g < Nq; ++g) {
        double w = 1.0;
        for (int r = 0; r < d; ++r) w *= t.gw1[digit(g, q1, r)];
        t.wq[g] = w;
        for (int j = 0; j < Np; ++j) {
            double v = 1.0;
            for (int r = 0; r < d; ++r) v *= B[(size_t)digit(g, q1, r) * n1 + digit(j, n1, r)];
            t.phi[(size_t)g * Np + j] = v;
            for (int k = 0; k < d; ++k) {
                double dv = 1.0;
                for (int r = 0; r < d; ++r) {
                    const std::vector<double>& T = (r == k) ? Dd : B;
                    dv *= T[(size_t)digit(g, q1, r) * n1 + digit(j, n1, r)];
                }
                t.dphi[((size_t)k * Nq + g) * Np + j] = dv;
            }
        }
    }
    // faces: face f = 2 r + side, local coordinates = remaining directions ascending
    t.mu.assign((size_t)Nfq * Nfp, 0.0);
    t.wf.assign(Nfq, 0.0);
    for (int s = 0; s < Nfq; ++s) {
        double w = 1.0;
        for (int a = 0; a < d - 1; ++a) w *= t.gw1[digit(s, q1, a)];
        t.wf[s] = w;
        for (int l = 0; l < Nfp; ++l) {
            double v = 1.0;
            for (int a = 0; a < d - 1; ++a) v *= B[(size_t)digit(s, q1, a) * n1 + digit(l, n1, a)];
            t.mu[(size_t)s * Nfp + l] = v;
        }
    }
    t.fnode.assign((size_t)nf * Nfp, 0);
    for (int f = 0; f < nf; ++f) {
        int r = f / 2, side = f % 2;
        for (int l = 0; l < Nfp; ++l) {
            int node = 0, a = 0, stride = 1;
            for (int k = 0; k < d; ++k) {
                int dk = (k == r) ? (side ? p : 0) : digit(l, n1, a++);
                node += dk * stride;
                stride *= n1;
            }
            t.fnode[(size_t)f * Nfp + l] = node;
        }
    }
    t.node_face.assign((size_t)Np * d, -1);
    for (int f = 0; f < nf; ++f)
        for (int l = 0; l < Nfp; ++l) {
            int j = t.fnode[(size_t)f * Nfp + l];
            for (int k = 0; k < d; ++k)
                if (t.node_face[(size_t)j * d + k] < 0) { t.node_face[(size_t)j * d + k] = f * Nfp + l; break; }
        }
    // element basis at face points (dense, for derived tables)
    std::vector<double> phif((size_t)nf * Nfq * Np, 0.0);
    for (int f = 0; f < nf; ++f)
        for (int s = 0; s < Nfq; ++s)
            for (int l = 0; l < Nfp; ++l)
                phif[((size_t)f * Nfq + s) * Np + t.fnode[(size_t)f * Nfp + l]] = t.mu[(size_t)s * Nfp + l];
    // mass matrices
    t.mhat.assign((size_t)Np * Np, 0.0);
    for (int i = 0; i < Np; ++i)
        for (int j = 0; j < Np; ++j) {
            double s = 0.0;
            for (int g = 0; g < Nq; ++g) s += t.wq[g] * t.phi[(size_t)g * Np + i] * t.phi[(size_t)g * Np + j];
            t.mhat[(size_t)i * Np + j] = s;
        }
    t.mf.assign((size_t)Nfp * Nfp, 0.0);
    for (int i = 0; i < Nfp; ++i)
        for (int j = 0; j < Nfp; ++j) {
            double s = 0.0;
            for (int q = 0; q < Nfq; ++q) s += t.wf[q] * t.mu[(size_t)q * Nfp + i] * t.mu[(size_t)q * Nfp + j];
            t.mf[(size_t)i * Nfp + j] = s;
        }
    std::vector<double> minv;
    invert(t.mhat, Np, minv);
    // Mhat^{-1} Chat_r, Chat_r[i][j] = sum_g w d_r phi_i phi_j
    t.minv_c.assign((size_t)d * Np * Np, 0.0);
    std::vector<double> C((size_t)Np * Np);
    for (int r = 0; r < d; ++r) {
        for (int i = 0; i < Np; ++i)
            for (int j = 0; j < Np; ++j) {
                double s = 0.0;
                for (int g = 0; g < Nq; ++g)
                    s += t.wq[g] * t.dphi[((size_t)r * Nq + g) * Np + i] * t.phi[(size_t)g * Np + j];
                C[(size_t)i * Np + j] = s;
            }
        for (int i = 0; i < Np; ++i)
            for (int j = 0; j < Np; ++j) {
                double s = 0.0;
                for (int k = 0; k < Np; ++k) s += minv[(size_t)i * Np + k] * C[(size_t)k * Np + j];
                t.minv_c[((size_t)r * Np + i) * Np + j] = s;
            }
    }
    // Mhat^{-1} Ehat_f, Ehat_f[i][l] = sum_s wf phi_i(s) mu_l(s)
    t.minv_e.assign((size_t)nf * Np * Nfp, 0.0);
    std::vector<double> Ef((size_t)Np * Nfp);
    for (int f = 0; f < nf; ++f) {
        for (int i = 0; i < Np; ++i)
            for (int l = 0; l < Nfp; ++l) {
                double s = 0.0;
                for (int q = 0; q < Nfq; ++q)
                    s += t.wf[q] * phif[((size_t)f * Nfq + q) * Np + i] * t.mu[(size_t)q * Nfp + l];
                Ef[(size_t)i * Nfp + l] = s;
            }
        for (int i = 0; i < Np; ++i)
            for (int l = 0; l < Nfp; ++l) {
                double s = 0.0;
                for (int k = 0; k < Np; ++k) s += minv[(size_t)i * Np + k] * Ef[(size_t)k * Nfp + l];
                t.minv_e[((size_t)f * Np + i) * Nfp + l] = s;
            }
    }
    // values at quadrature points
    t.psi.assign((size_t)d * Nq * Np, 0.0);
    for (int r = 0; r < d; ++r)
        for (int g = 0; g < Nq; ++g)
            for (int j = 0; j < Np; ++j) {
                double s = 0.0;
                for (int k = 0; k < Np; ++k)
                    s += t.phi[(size_t)g * Np + k] * t.minv_c[((size_t)r * Np + k) * Np + j];
                t.psi[((size_t)r * Nq + g) * Np + j] = s;
            }
    t.theta.assign((size_t)nf * Nq * Nfp, 0.0);
    for (int f = 0; f < nf; ++f)
        for (int g = 0; g < Nq; ++g)
            for (int l = 0; l < Nfp; ++l) {
                double s = 0.0;
                for (int k = 0; k < Np; ++k)
                    s += t.phi[(size_t)g * Np + k] * t.minv_e[((size_t)f * Np + k) * Nfp + l];
                t.theta[((size_t)f * Nq + g) * Nfp + l] = s;
            }
    t.psi_f.assign((size_t)nf * d * Nfq * Np, 0.0);
    for (int f = 0; f < nf; ++f)
        for (int r = 0; r < d; ++r)
            for (int q = 0; q < Nfq; ++q)
                for (int j = 0; j < Np; ++j) {
                    double s = 0.0;
                    for (int k = 0; k < Np; ++k)
                        s += phif[((size_t)f * Nfq + q) * Np + k] * t.minv_c[((size_t)r * Np + k) * Np + j];
                    t.psi_f[(((size_t)f * d + r) * Nfq + q) * Np + j] = s;
                }
    t.theta_f.assign((size_t)nf * nf * Nfq * Nfp, 0.0);
    for (int f = 0; f < nf; ++f)
        for (int f2 = 0; f2 < nf; ++f2)
            for (int q = 0; q < Nfq; ++q)
                for (int l = 0; l < Nfp; ++l) {
                    double s = 0.0;
                    for (int k = 0; k < Np; ++k)
                        s += phif[((size_t)f * Nfq + q) * Np + k] * t.minv_e[((size_t)f2 * Np + k) * Nfp + l];
                    t.theta_f[(((size_t)f * nf + f2) * Nfq + q) * Nfp + l] = s;
                }
}

}  // namespace hdg
