// FP64 kernels of the HDG linearize + condense path, templated on (d, p).
//
// Per element K the path forms the bordered matrix
//
//     [ At  Bt  Rt ]     At = A_uu - A_uq A_qq^{-1} A_qu      (n_u x n_u)
//     [ Ct  Dt  Rh ]     Bt = B_u  - A_uq A_qq^{-1} B_q       (n_u x t)
//                        Ct = C_u  - C_q  A_qq^{-1} A_qu      (t x n_u)
//                        Dt = D    - C_q  A_qq^{-1} B_q       (t x t)
//
// i.e. the element system of eq. newton-local-block with the gradient block
// eliminated exactly (A_qq = I (x) M_K is the mass matrix and R_q is linear,
// eq. hdg-grad), and eliminates its first n_u columns by Gaussian elimination
// with partial pivoting restricted to the first n_u rows.  The trailing block
// is then S^K = Dt - Ct At^{-1} Bt = D - C A^{-1} B and the last column
// -g^K (eq. schur-trace); the first n_u rows keep [U | L^{-1} P Bt | L^{-1} P Rt]
// for the recovery of eq. local-elimination.
//
// The right-hand-side column uses the fluxes at the lifted gradient
// Q_lift(U, Uhat) = Q - A_qq^{-1} R_q: R_u and R_uhat are affine in Q, so
// R_u(Q_lift) = R_u - A_uq A_qq^{-1} R_q exactly.
#pragma once

#include <climits>

#include "common.h"
#include "physics.cuh"
#include "tc_util.cuh"
#include "tma.h"

namespace hdg {

// per-element geometry record: detJ, Jinv[d][d] (d xi_r / d x_k), NW[nf][d]
template <int D> struct Geo { static constexpr int N = 1 + D * D + 2 * D * D; };

// Storage of the bordered matrix [[At, Bt, Rt], [Ct, Dt, Rh]] of each element as
// region views: base pointer, element stride and row stride.  Interior rows are
// indexed by the global element, trace rows by the element's index in the chunk.
// The FP64 form keeps one row-major matrix per element (all views alias it);
// the mixed form keeps At and the right-hand sides in FP64 and Bt, Ct, Dt in TL.
template <class TL>
struct Regions {
    double* a11; int64_t a11_es, a11_rs;   // At  [n_u][n_u]
    TL* a12; int64_t a12_es, a12_rs;       // Bt  [n_u][t]
    TL* a21; int64_t a21_es, a21_rs;       // Ct  [t][n_u]   (chunk-local)
    TL* a22; int64_t a22_es, a22_rs;       // Dt  [t][t]     (chunk-local)
    double* rt; int64_t rt_es, rt_rs;      // Rt  [n_u]
    double* rb; int64_t rb_es, rb_rs;      // Rh  [t]        (chunk-local)
};

// views of the FP64 form's single row-major bordered matrix (row stride LD)
template <class C>
inline Regions<double> fp64_regions(double* top, double* bot) {
    constexpr int64_t NU = C::NU, NT = C::NT, LD = C::LD, NC = C::NC;
    Regions<double> R;
    R.a11 = top;           R.a11_es = NU * LD; R.a11_rs = LD;
    R.a12 = top + NU;      R.a12_es = NU * LD; R.a12_rs = LD;
    R.a21 = bot;           R.a21_es = NT * LD; R.a21_rs = LD;
    R.a22 = bot + NU;      R.a22_es = NT * LD; R.a22_rs = LD;
    R.rt = top + NC - 1;   R.rt_es = NU * LD;  R.rt_rs = LD;
    R.rb = bot + NC - 1;   R.rb_es = NT * LD;  R.rb_rs = LD;
    return R;
}

// ----------------------------------------------------------------------------
// A0 + A1: gather, interpolation, fluxes and their Jacobians at quadrature points
// ----------------------------------------------------------------------------
struct PointArgs {
    const double* U; const double* Q; const double* UH; const double* Ustar; const double* nu;
    double dt, a_ii;
    PhysT<double> ph;        // residual terms (FP64)
    PhysT<float> phf;        // Jacobian terms of the mixed form
    double tau;
    DeviceTables tab;
    const double* geo;
    const int32_t* e2f; const int32_t* perm;
    double* rt; int64_t rt_es, rt_rs;      // right-hand side, interior rows
    double* rb; int64_t rb_es, rb_rs;      // right-hand side, trace rows (chunk-local)
    void* vcoef; void* fcoef;   // Jacobian coefficients, in the form's Jacobian type
    double* dq0;
    const int32_t* ftag;        // [E][nf] boundary tag of each element face (0 interior / periodic)
    const double* ub;           // [m] boundary state of tag-1 faces
    const double* ubf;          // [F][m][Nfp] nodal tag-1 boundary data (canonical order), or NULL
    double ew;                  // wall internal energy c_v T_w of tag-3 faces
    int tau_mode;               // 0: constant tau; 1: state-dependent tau(uhat) (stab_tau)
    double* taup;               // [chunk][nf][Nfq] tau at the face points (tau_mode 1), for the face terms
    int64_t e0;
};

// Boundary form bhat_a at one face quadrature point, scaled by w_s |J_s| like
// the numerical flux fh = w_s |J_s| fhat_a it may take rows from (Sec. 2.2;
// the forms are readings):
//   tag 1 far-field / supersonic inflow   uhat - u_b
//   tag 2 supersonic outflow              uhat - u      (interior state extrapolated)
//   tag 3 isothermal no-slip wall         [fhat_rho; uhat_rhov; uhat_rhoE - uhat_rho e_w]
//   tag 4 adiabatic no-slip wall          [fhat_rho; uhat_rhov; fhat_rhoE]
template <int M>
__device__ __forceinline__ double boundary_form(int tag, int a, double fh, double wn, const double* u,
                                                const double* uh, double ub_a, double ew) {
    switch (tag) {
        case 1: return wn * (uh[a] - ub_a);
        case 2: return wn * (uh[a] - u[a]);
        case 3: return a == 0 ? fh : (a == M - 1 ? wn * (uh[a] - uh[0] * ew) : wn * uh[a]);
        case 4: return (a == 0 || a == M - 1) ? fh : wn * uh[a];
        default: return fh;
    }
}

// trace rows of a boundary face that are copies of the numerical-flux rows
template <int M>
__device__ __forceinline__ bool boundary_row_is_flux(int tag, int a) {
    return tag == 0 || (tag == 3 && a == 0) || (tag == 4 && (a == 0 || a == M - 1));
}

// u_b,a at face quadrature point s of local face f of element e (tag-1 faces)
template <int NF, int M, int NFP>
__device__ __forceinline__ double boundary_state(const double* ub, const double* ubf, const int32_t* e2f,
                                                 const int32_t* perm, const double* mu, int64_t e, int f, int s,
                                                 int a) {
    if (!ubf) return ub[a];
    const int64_t F = e2f[e * NF + f];
    double v = 0.0;
    for (int lam = 0; lam < NFP; ++lam)
        v += mu[s * NFP + lam] * ubf[(F * M + a) * NFP + perm[(e * NF + f) * NFP + lam]];
    return v;
}

template <class S> __device__ __forceinline__ const PhysT<S>& jac_phys(const PointArgs& A);
template <> __device__ __forceinline__ const PhysT<double>& jac_phys<double>(const PointArgs& A) { return A.ph; }
template <> __device__ __forceinline__ const PhysT<float>& jac_phys<float>(const PointArgs& A) { return A.phf; }

template <class C>
constexpr int point_smem_doubles() {
    return C::NU + 2 * C::NQV + C::NP + 2 * C::NT + C::D * C::M * C::NQ + 2 * C::NF * C::M * C::NFQ;
}

template <class C, int NTH, class TJ>
__global__ void __launch_bounds__(NTH) k_point(PointArgs A) {
    constexpr int D = C::D, M = C::M, NP = C::NP, NQ = C::NQ, NF = C::NF, NFP = C::NFP, NFQ = C::NFQ;
    constexpr int NU = C::NU, NQV = C::NQV, NT = C::NT, NCOEF = C::NCOEF;
    constexpr int GEO = Geo<D>::N;
    const int tid = threadIdx.x;
    const int64_t el = blockIdx.x, e = A.e0 + el;
    extern __shared__ double sm[];
    double* sU = sm;                     // [m][Np]
    double* sQ = sU + NU;                // [d][m][Np]
    double* sQL = sQ + NQV;              // lifted gradient [d][m][Np]
    double* sNu = sQL + NQV;             // [Np]
    double* sUH = sNu + NP;              // [nf][m][Nfp] element-local face order
    double* sFres = sUH + NT;            // [d][m][Nq]
    double* sFH = sFres + D * M * NQ;    // [nf][m][Nfq]
    double* sRh = sFH + NF * M * NFQ;    // [nf][m][Nfp]
    double* sFB = sRh + NT;              // [nf][m][Nfq] boundary form bhat (boundary faces)
    __shared__ double geo[GEO];
    const DeviceTables& T = A.tab;

    for (int i = tid; i < NU; i += NTH) sU[i] = A.U[e * NU + i];
    for (int i = tid; i < NQV; i += NTH) sQ[i] = A.Q[e * NQV + i];
    for (int i = tid; i < NP; i += NTH) sNu[i] = A.nu ? A.nu[e * NP + i] : 0.0;
    for (int i = tid; i < NT; i += NTH) {
        int f = i / (M * NFP), rem = i - f * M * NFP, a = rem / NFP, l = rem - a * NFP;
        int64_t F = A.e2f[e * NF + f];
        int k = A.perm[(e * NF + f) * NFP + l];
        sUH[i] = A.UH[(F * M + a) * NFP + k];
    }
    for (int i = tid; i < GEO; i += NTH) geo[i] = A.geo[e * GEO + i];
    __syncthreads();
    const double detJ = geo[0];
    const double* Jinv = geo + 1;
    const double* NW = geo + 1 + D * D;

    // lifted gradient at the nodes: Q_lift = -L U + Lambda Uhat (A_qq^{-1} applied)
    for (int idx = tid; idx < M * NP; idx += NTH) {
        int a = idx / NP, i = idx - a * NP;
        double t[D], ef[NF];
        for (int r = 0; r < D; ++r) {
            double s = 0.0;
            const double* mc = T.minv_c + ((size_t)r * NP + i) * NP;
            for (int j = 0; j < NP; ++j) s += mc[j] * sU[a * NP + j];
            t[r] = s;
        }
        for (int f = 0; f < NF; ++f) {
            double s = 0.0;
            const double* me = T.minv_e + ((size_t)f * NP + i) * NFP;
            for (int l = 0; l < NFP; ++l) s += me[l] * sUH[(f * M + a) * NFP + l];
            ef[f] = s;
        }
        for (int l = 0; l < D; ++l) {
            double ql = 0.0;
            for (int r = 0; r < D; ++r) ql -= Jinv[r * D + l] * t[r];
            for (int f = 0; f < NF; ++f) ql += NW[f * D + l] / detJ * ef[f];
            int o = (l * M + a) * NP + i;
            sQL[o] = ql;
            A.dq0[e * NQV + o] = ql - sQ[o];
        }
    }
    __syncthreads();

    const PhysT<double>& ph = A.ph;
    const PhysT<TJ>& pj = jac_phys<TJ>(A);
    TJ* vc = reinterpret_cast<TJ*>(A.vcoef) + el * (size_t)(M * M * D * NCOEF * NQ);
    TJ Jj[D * D], NWj[NF * D];
    for (int i = 0; i < D * D; ++i) Jj[i] = (TJ)Jinv[i];
    for (int i = 0; i < NF * D; ++i) NWj[i] = (TJ)(NW[i] / detJ);
    // volume points
    for (int g = tid; g < NQ; g += NTH) {
        double u[M], q[M][D], ql[M][D], nuv = 0.0;
        for (int a = 0; a < M; ++a) { u[a] = 0.0; for (int l = 0; l < D; ++l) { q[a][l] = 0.0; ql[a][l] = 0.0; } }
        for (int j = 0; j < NP; ++j) {
            double w = T.phi[g * NP + j];
            nuv += w * sNu[j];
            for (int a = 0; a < M; ++a) {
                u[a] += w * sU[a * NP + j];
                for (int l = 0; l < D; ++l) {
                    q[a][l] += w * sQ[(l * M + a) * NP + j];
                    ql[a][l] += w * sQL[(l * M + a) * NP + j];
                }
            }
        }
        const double wJ = -A.dt * T.wq[g] * detJ;
        {
            double Fc[M][D], Fv[M][D];
            conv_flux<D, double, double>(u, ph, Fc);
            visc_flux<D, double, double>(u, ql, nuv, ph, Fv);
            for (int r = 0; r < D; ++r)
                for (int a = 0; a < M; ++a) {
                    double s = 0.0;
                    for (int k = 0; k < D; ++k) s += Jinv[r * D + k] * (Fc[a][k] - Fv[a][k]);
                    sFres[(r * M + a) * NQ + g] = wJ * s;
                }
        }
        // Jacobian coefficients in TJ
        TJ uj[M], qj[M][D];
        for (int a = 0; a < M; ++a) { uj[a] = (TJ)u[a]; for (int l = 0; l < D; ++l) qj[a][l] = (TJ)q[a][l]; }
        const TJ nuj = (TJ)nuv, wJj = (TJ)wJ;
        for (int b = 0; b < M; ++b) {
            DirT<TJ> ud[M];
            for (int a = 0; a < M; ++a) ud[a] = {uj[a], a == b ? TJ(1) : TJ(0)};
            DirT<TJ> Fc[M][D], Fv[M][D];
            conv_flux<D, DirT<TJ>, TJ>(ud, pj, Fc);
            visc_flux<D, DirT<TJ>, TJ>(ud, qj, nuj, pj, Fv);
            for (int a = 0; a < M; ++a)
                for (int r = 0; r < D; ++r) {
                    TJ s = 0;
                    for (int k = 0; k < D; ++k) s += Jj[r * D + k] * (Fc[a][k].t - Fv[a][k].t);
                    vc[((((size_t)a * M + b) * D + r) * NCOEF + 0) * NQ + g] = wJj * s;
                }
        }
        for (int b = 0; b < M; ++b) {
            TJ cq[D][M][D];
            for (int l = 0; l < D; ++l) {
                TJ qe[M][D];
                for (int a = 0; a < M; ++a) for (int k = 0; k < D; ++k) qe[a][k] = (a == b && k == l) ? TJ(1) : TJ(0);
                TJ Fv[M][D];
                visc_flux<D, TJ, TJ>(uj, qe, nuj, pj, Fv);
                for (int r = 0; r < D; ++r)
                    for (int a = 0; a < M; ++a) {
                        TJ s = 0;
                        for (int k = 0; k < D; ++k) s += Jj[r * D + k] * Fv[a][k];
                        cq[r][a][l] = -wJj * s;
                    }
            }
            for (int a = 0; a < M; ++a)
                for (int r = 0; r < D; ++r) {
                    TJ* o = vc + ((((size_t)a * M + b) * D + r) * NCOEF) * NQ + g;
                    for (int r2 = 0; r2 < D; ++r2) {
                        TJ s = 0;
                        for (int l = 0; l < D; ++l) s += cq[r][a][l] * Jj[r2 * D + l];
                        o[(1 + r2) * NQ] = s;
                    }
                    for (int f = 0; f < NF; ++f) {
                        TJ s = 0;
                        for (int l = 0; l < D; ++l) s += cq[r][a][l] * NWj[f * D + l];
                        o[(1 + D + f) * NQ] = s;
                    }
                }
        }
    }
    // face points
    TJ* fc = reinterpret_cast<TJ*>(A.fcoef) + el * (size_t)(NF * M * M * NCOEF * NFQ);
    for (int fs = tid; fs < NF * NFQ; fs += NTH) {
        const int f = fs / NFQ, s = fs - f * NFQ;
        double u[M], uh[M], q[M][D], ql[M][D], nuv = 0.0;
        for (int a = 0; a < M; ++a) { u[a] = 0.0; uh[a] = 0.0; for (int l = 0; l < D; ++l) { q[a][l] = 0.0; ql[a][l] = 0.0; } }
        for (int lam = 0; lam < NFP; ++lam) {
            double w = T.mu[s * NFP + lam];
            int j = T.fnode[f * NFP + lam];
            nuv += w * sNu[j];
            for (int a = 0; a < M; ++a) {
                u[a] += w * sU[a * NP + j];
                uh[a] += w * sUH[(f * M + a) * NFP + lam];
                for (int l = 0; l < D; ++l) {
                    q[a][l] += w * sQ[(l * M + a) * NP + j];
                    ql[a][l] += w * sQL[(l * M + a) * NP + j];
                }
            }
        }
        const double* nw = NW + f * D;
        double nrm = 0.0;
        for (int k = 0; k < D; ++k) nrm += nw[k] * nw[k];
        nrm = sqrt(nrm);
        const double ws = T.wf[s];
        double nh[D];
        for (int k = 0; k < D; ++k) nh[k] = nw[k] / nrm;
        const double hinv = A.tau_mode ? 1.0 / pow(double(1 << D) * detJ, 1.0 / D) : 0.0;   // |K|^{-1/d}
        const double tau_s = A.tau_mode ? stab_tau<D, double, double>(uh, nh, hinv, ph) : A.tau;
        if (A.taup) A.taup[(el * NF + f) * NFQ + s] = tau_s;
        {
            double Fc[M][D], Fv[M][D];
            conv_flux<D, double, double>(uh, ph, Fc);
            visc_flux<D, double, double>(uh, ql, nuv, ph, Fv);
            const int tag = A.ftag ? A.ftag[e * NF + f] : 0;
            for (int a = 0; a < M; ++a) {
                double fn = 0.0;
                for (int k = 0; k < D; ++k) fn += (Fc[a][k] - Fv[a][k]) * nw[k];
                const double fh = ws * (fn + nrm * tau_s * (u[a] - uh[a]));
                sFH[(f * M + a) * NFQ + s] = fh;
                const double ub_a = tag == 1 ? boundary_state<NF, M, NFP>(A.ub, A.ubf, A.e2f, A.perm, T.mu, e, f, s, a) : 0.0;
                sFB[(f * M + a) * NFQ + s] = boundary_form<M>(tag, a, fh, ws * nrm, u, uh, ub_a, A.ew);
            }
        }
        TJ uhj[M], qj[M][D], nwj[D];
        for (int a = 0; a < M; ++a) { uhj[a] = (TJ)uh[a]; for (int l = 0; l < D; ++l) qj[a][l] = (TJ)q[a][l]; }
        for (int k = 0; k < D; ++k) nwj[k] = (TJ)nw[k];
        const TJ nuj = (TJ)nuv, wsj = (TJ)ws, taun = (TJ)(nrm * tau_s);
        TJ nhj[D];
        for (int k = 0; k < D; ++k) nhj[k] = (TJ)nh[k];
        for (int b = 0; b < M; ++b) {
            DirT<TJ> ud[M];
            for (int a = 0; a < M; ++a) ud[a] = {uhj[a], a == b ? TJ(1) : TJ(0)};
            DirT<TJ> Fc[M][D], Fv[M][D];
            conv_flux<D, DirT<TJ>, TJ>(ud, pj, Fc);
            visc_flux<D, DirT<TJ>, TJ>(ud, qj, nuj, pj, Fv);
            // d tau / d uhat_b (state-dependent stabilization): (u_a - uhat_a) |nw| d tau / d uhat_b
            const TJ dtau = A.tau_mode ? (TJ)nrm * stab_tau<D, DirT<TJ>, TJ>(ud, nhj, (TJ)hinv, pj).t : TJ(0);
            for (int a = 0; a < M; ++a) {
                TJ fn = 0;
                for (int k = 0; k < D; ++k) fn += (Fc[a][k].t - Fv[a][k].t) * nwj[k];
                if (a == b) fn -= taun;
                fn += ((TJ)u[a] - uhj[a]) * dtau;
                fc[((((size_t)f * M + a) * M + b) * NCOEF + 0) * NFQ + s] = wsj * fn;
            }
        }
        for (int b = 0; b < M; ++b) {
            TJ qh[M][D];
            for (int l = 0; l < D; ++l) {
                TJ qe[M][D];
                for (int a = 0; a < M; ++a) for (int k = 0; k < D; ++k) qe[a][k] = (a == b && k == l) ? TJ(1) : TJ(0);
                TJ Fv[M][D];
                visc_flux<D, TJ, TJ>(uhj, qe, nuj, pj, Fv);
                for (int a = 0; a < M; ++a) {
                    TJ fn = 0;
                    for (int k = 0; k < D; ++k) fn += Fv[a][k] * nwj[k];
                    qh[a][l] = -wsj * fn;
                }
            }
            for (int a = 0; a < M; ++a) {
                TJ* o = fc + ((((size_t)f * M + a) * M + b) * NCOEF) * NFQ + s;
                for (int r2 = 0; r2 < D; ++r2) {
                    TJ t = 0;
                    for (int l = 0; l < D; ++l) t += qh[a][l] * Jj[r2 * D + l];
                    o[(1 + r2) * NFQ] = t;
                }
                for (int f2 = 0; f2 < NF; ++f2) {
                    TJ t = 0;
                    for (int l = 0; l < D; ++l) t += qh[a][l] * NWj[f2 * D + l];
                    o[(1 + D + f2) * NFQ] = t;
                }
            }
        }
    }
    __syncthreads();
    // right-hand-side column: Rh (trace rows) then Rt (interior rows)
    double* rbe = A.rb + el * A.rb_es;
    for (int idx = tid; idx < NT; idx += NTH) {
        int f = idx / (M * NFP), rem = idx - f * M * NFP, a = rem / NFP, l = rem - a * NFP;
        double s = 0.0, sb = 0.0;
        for (int q = 0; q < NFQ; ++q) {
            s += T.mu[q * NFP + l] * sFH[(f * M + a) * NFQ + q];
            sb += T.mu[q * NFP + l] * sFB[(f * M + a) * NFQ + q];
        }
        sRh[idx] = s;
        const bool bnd = A.ftag && A.ftag[e * NF + f] != 0;
        rbe[idx * A.rb_rs] = bnd ? sb : s;
    }
    __syncthreads();
    double* rte = A.rt + e * A.rt_es;
    for (int idx = tid; idx < NU; idx += NTH) {
        int a = idx / NP, i = idx - a * NP;
        double mass = 0.0;
        for (int j = 0; j < NP; ++j) mass += T.mhat[i * NP + j] * (sU[a * NP + j] - A.Ustar[e * NU + a * NP + j]);
        double s = mass * detJ / A.a_ii;
        for (int r = 0; r < D; ++r)
            for (int g = 0; g < NQ; ++g) s += T.dphi[((size_t)r * NQ + g) * NP + i] * sFres[(r * M + a) * NQ + g];
        for (int k = 0; k < D; ++k) {
            int nfc = T.node_face[i * D + k];
            if (nfc < 0) continue;
            int f = nfc / NFP, l = nfc - f * NFP;
            s += A.dt * sRh[(f * M + a) * NFP + l];
        }
        rte[idx * A.rt_rs] = s;
    }
}

// ----------------------------------------------------------------------------
// A2: contraction of the coefficients with the basis tables into the blocks
// ----------------------------------------------------------------------------
template <class TL>
struct BlkArgs {
    const void* vcoef; const void* fcoef;   // Jacobian coefficients in the accumulation type
    const int32_t* ftag;                    // [E][nf] or NULL
    const double* geo;
    DeviceTables tab;
    Regions<TL> R;
    double dt, a_ii, tau;
    double ew;                              // wall internal energy of tag-3 faces
    const double* taup;                     // [chunk][nf][Nfq] per-point tau (state-dependent), or NULL
    int64_t e0;
};

template <class C, int TY, int TX, int KC>
struct BlkShape {
    static constexpr int NCB = C::NP + C::NF * C::NFP;
    static constexpr int NTH = TY * TX;
    // register tiles when the output tile divides evenly; otherwise a flat
    // thread -> output map (two shared loads per DFMA are free next to the FP64 pipe)
    static constexpr bool FLAT = (C::NP % TY) != 0 || (NCB % TX) != 0;
    static constexpr int TM = FLAT ? 1 : C::NP / TY, TN = FLAT ? 1 : NCB / TX;
    static constexpr int SLOTS = (C::NP * NCB + NTH - 1) / NTH;
    static constexpr int NPP = C::NP, NCBP = NCB;
    static constexpr int main_smem = KC * (NPP + NCBP + C::NCOEF);
    static constexpr int face_smem = C::NCOEF * C::NFQ + C::NFQ * NCB;
    static constexpr int smem = main_smem > face_smem ? main_smem : face_smem;
    // FP32 form: the face terms of the interior block are summed over the faces in a
    // [Np][Np] shared tile and added to the FP64 block once
    static constexpr int face_acc_smem = face_smem + C::NP * C::NP;
    static constexpr int smem_f32 = main_smem > face_acc_smem ? main_smem : face_acc_smem;
};

// VOL = false skips the volume contraction (done on tensor cores by
// k_blocks_tc in the mixed form) and adds only the face terms.
template <class C, int TY, int TX, int KC, class TA, class TL, bool VOL = true>
__global__ void __launch_bounds__(TY * TX) k_blocks(BlkArgs<TL> A) {
    constexpr int D = C::D, M = C::M, NP = C::NP, NQ = C::NQ, NF = C::NF, NFP = C::NFP, NFQ = C::NFQ;
    constexpr int NCOEF = C::NCOEF;
    using S = BlkShape<C, TY, TX, KC>;
    constexpr int NCB = S::NCB, TM = S::TM, TN = S::TN, NPP = S::NPP, NCBP = S::NCBP;
    constexpr int K = D * NQ, NTH = TY * TX;
    constexpr int GEO = Geo<D>::N;
    const int tid = threadIdx.x, ty = tid / TX, tx = tid - ty * TX;
    const int64_t bid = blockIdx.x;
    const int b = (int)(bid % M), a = (int)((bid / M) % M);
    const int64_t el = bid / (M * M), e = A.e0 + el;
    const DeviceTables& T = A.tab;
    extern __shared__ double sm_raw[];
    TA* sm = reinterpret_cast<TA*>(sm_raw);
    TA* As = sm;
    TA* Bs = As + KC * NPP;
    TA* Cs = Bs + KC * NCBP;
    const TA* cf = reinterpret_cast<const TA*>(A.vcoef) + (((size_t)el * M + a) * M + b) * (size_t)(D * NCOEF * NQ);
    // reference tables in the accumulation type
    constexpr bool F32 = sizeof(TA) == 4;
    const TA* tphi = F32 ? (const TA*)T.fphi : (const TA*)T.phi;
    const TA* tdphi = F32 ? (const TA*)T.fdphi : (const TA*)T.dphi;
    const TA* tpsi = F32 ? (const TA*)T.fpsi : (const TA*)T.psi;
    const TA* ttheta = F32 ? (const TA*)T.ftheta : (const TA*)T.theta;
    const TA* tpsif = F32 ? (const TA*)T.fpsi_f : (const TA*)T.psi_f;
    const TA* tthetaf = F32 ? (const TA*)T.ftheta_f : (const TA*)T.theta_f;
    const TA* tmu = F32 ? (const TA*)T.fmu : (const TA*)T.mu;
    const TA* tmf = F32 ? (const TA*)T.fmf : (const TA*)T.mf;

    constexpr bool FLAT = S::FLAT;
    constexpr int SL = FLAT ? S::SLOTS : TM * TN;
    TA acc[SL];
    int ri[SL], ci[SL];
#pragma unroll
    for (int s = 0; s < SL; ++s) {
        acc[s] = 0.0;
        if (FLAT) {
            int idx = tid + NTH * s;
            ri[s] = idx < NP * NCB ? idx / NCB : -1;
            ci[s] = idx < NP * NCB ? idx - (idx / NCB) * NCB : 0;
        } else {
            ri[s] = ty + TY * (s / TN);
            ci[s] = tx + TX * (s % TN);
        }
    }

    for (int k0 = 0; VOL && k0 < K; k0 += KC) {
        const int kc = min(KC, K - k0);
        for (int idx = tid; idx < kc * NCOEF; idx += NTH) {
            int kk = idx / NCOEF, c = idx - kk * NCOEF, k = k0 + kk, r = k / NQ, g = k - r * NQ;
            Cs[idx] = cf[(r * NCOEF + c) * NQ + g];
        }
        for (int idx = tid; idx < kc * NPP; idx += NTH) As[idx] = tdphi[(size_t)k0 * NP + idx];
        __syncthreads();
        for (int idx = tid; idx < kc * NCBP; idx += NTH) {
            int kk = idx / NCBP, c = idx - kk * NCBP;
            int k = k0 + kk, r = k / NQ, g = k - r * NQ;
            const TA* cc = Cs + kk * NCOEF;
            TA v;
            if (c < NP) {
                v = cc[0] * tphi[g * NP + c];
                for (int r2 = 0; r2 < D; ++r2) v -= cc[1 + r2] * tpsi[((size_t)r2 * NQ + g) * NP + c];
            } else {
                int c2 = c - NP, f = c2 / NFP, l = c2 - f * NFP;
                v = cc[1 + D + f] * ttheta[((size_t)f * NQ + g) * NFP + l];
            }
            Bs[idx] = v;
        }
        __syncthreads();
        if (FLAT) {
            for (int kk = 0; kk < kc; ++kk) {
#pragma unroll
                for (int s = 0; s < SL; ++s)
                    if (ri[s] >= 0) acc[s] = fma(As[kk * NPP + ri[s]], Bs[kk * NCBP + ci[s]], acc[s]);
            }
        } else {
            for (int kk = 0; kk < kc; ++kk) {
                TA av[TM], bv[TN];
#pragma unroll
                for (int ii = 0; ii < TM; ++ii) av[ii] = As[kk * NPP + ty + TY * ii];
#pragma unroll
                for (int jj = 0; jj < TN; ++jj) bv[jj] = Bs[kk * NCBP + tx + TX * jj];
#pragma unroll
                for (int ii = 0; ii < TM; ++ii)
#pragma unroll
                    for (int jj = 0; jj < TN; ++jj) acc[ii * TN + jj] = fma(av[ii], bv[jj], acc[ii * TN + jj]);
            }
        }
        __syncthreads();
    }

    const double* G = A.geo + e * GEO;
    const double detJ = G[0];
    double* A11 = A.R.a11 + e * A.R.a11_es;
    TL* A12 = A.R.a12 + e * A.R.a12_es;
#pragma unroll
    for (int s = 0; s < SL; ++s) {
        const int i = ri[s], c = ci[s];
        if (!VOL || i < 0 || i >= NP || c >= NCB) continue;
        const int64_t row = a * NP + i;
        if (c < NP) {
            double v = (double)acc[s];
            if (a == b) v += detJ / A.a_ii * T.mhat[i * NP + c];
            A11[row * A.R.a11_rs + b * NP + c] = v;
        } else {
            int c2 = c - NP, f = c2 / NFP, l = c2 - f * NFP;
            A12[row * A.R.a12_rs + (f * M + b) * NFP + l] = (TL)acc[s];
        }
    }
    __syncthreads();

    // face terms: rows of Ct / Dt, and dt x the same rows added to At / Bt at the face nodes
    TL* A21 = A.R.a21 + el * A.R.a21_es;
    TL* A22 = A.R.a22 + el * A.R.a22_es;
    TA* Fc = sm;                           // [NCOEF][Nfq]
    TA* Tt = Fc + NCOEF * NFQ;             // [Nfq][NCB]
    constexpr bool FACC = sizeof(TA) == 4;  // FP32 form: sum the At face terms in shared memory
    TA* Acc = Tt + NFQ * NCB;              // [Np][Np] (FP32 form only)
    if (FACC) {
        for (int idx = tid; idx < NP * NP; idx += NTH) Acc[idx] = (TA)0;
        __syncthreads();
    }
    const double* NW = G + 1 + D * D;
    const double* Jg = G + 1;
    (void)Jg;
    __shared__ TA mft[NFP * NFP];          // state-dependent tau: face mass weighted by tau(s)
    for (int f = 0; f < NF; ++f) {
        const TA* fsrc = reinterpret_cast<const TA*>(A.fcoef) + ((((size_t)el * NF + f) * M + a) * M + b) * (size_t)(NCOEF * NFQ);
        for (int idx = tid; idx < NCOEF * NFQ; idx += NTH) Fc[idx] = fsrc[idx];
        if (A.taup)
            for (int idx = tid; idx < NFP * NFP; idx += NTH) {
                const int lam = idx / NFP, l = idx - lam * NFP;
                double w = 0.0;
                for (int q = 0; q < NFQ; ++q)
                    w += T.wf[q] * A.taup[(el * NF + f) * NFQ + q] * T.mu[q * NFP + lam] * T.mu[q * NFP + l];
                mft[idx] = (TA)w;
            }
        __syncthreads();
        for (int idx = tid; idx < NFQ * NCB; idx += NTH) {
            int s = idx / NCB, c = idx - s * NCB;
            TA v = 0;
            if (c < NP) {
                for (int r2 = 0; r2 < D; ++r2)
                    v -= Fc[(1 + r2) * NFQ + s] * tpsif[(((size_t)f * D + r2) * NFQ + s) * NP + c];
            } else {
                int c2 = c - NP, f2 = c2 / NFP, l2 = c2 - f2 * NFP;
                v = Fc[(1 + D + f2) * NFQ + s] * tthetaf[(((size_t)f * NF + f2) * NFQ + s) * NFP + l2];
                if (f2 == f) v += Fc[s] * tmu[s * NFP + l2];
            }
            Tt[idx] = v;
        }
        __syncthreads();
        double nrm = 0.0;
        for (int k = 0; k < D; ++k) nrm += NW[f * D + k] * NW[f * D + k];
        nrm = sqrt(nrm);
        const TA taun = (TA)(A.tau * nrm), dtt = (TA)A.dt;
        const int tag = A.ftag ? A.ftag[e * NF + f] : 0;
        // trace rows of a boundary face: copies of the numerical-flux rows, or algebraic in
        // (uhat, u) with d bhat_a / d uhat_b = cb * face mass and d bhat_a / d u_b = cu * face mass
        const bool flux_row = boundary_row_is_flux<M>(tag, a);
        const TA nrmt = (TA)nrm;
        TA cb = (a == b) ? (TA)1 : (TA)0, cu = (TA)0;
        if (tag == 3 && a == M - 1 && b == 0) cb = (TA)(-A.ew);
        if (tag == 2 && a == b) cu = (TA)(-1);
        for (int idx = tid; idx < NFP * NCB; idx += NTH) {
            int lam = idx / NCB, c = idx - lam * NCB;
            TA v = 0;
            for (int s = 0; s < NFQ; ++s) v += tmu[s * NFP + lam] * Tt[s * NCB + c];
            const int64_t trow = (f * M + a) * NFP + lam;
            const int64_t irow = a * NP + T.fnode[f * NFP + lam];
            if (c < NP) {
                TA vu = 0, vut = 0;                // face mass coupling of node c, if it lies on face f
                for (int k = 0; k < D; ++k) {
                    int nfc = T.node_face[c * D + k];
                    if (nfc >= 0 && nfc / NFP == f) {
                        vu = tmf[lam * NFP + (nfc - f * NFP)];
                        if (A.taup) vut = mft[lam * NFP + (nfc - f * NFP)];
                    }
                }
                if (a == b) v += A.taup ? nrmt * vut : taun * vu;
                const int col = b * NP + c;
                A21[trow * A.R.a21_rs + col] = flux_row ? (TL)v : (TL)(cu * nrmt * vu);
                if (FACC)   // one thread per (node, column) within a face; faces run one after another
                    Acc[T.fnode[f * NFP + lam] * NP + c] += dtt * v;
                else
                    A11[irow * A.R.a11_rs + col] += A.dt * (double)v;
            } else {
                int c2 = c - NP, f2 = c2 / NFP, l2 = c2 - f2 * NFP;
                const int col = (f2 * M + b) * NFP + l2;
                const TA vb = (f2 == f) ? cb * nrmt * tmf[lam * NFP + l2] : (TA)0;
                A22[trow * A.R.a22_rs + col] = flux_row ? (TL)v : (TL)vb;
                A12[irow * A.R.a12_rs + col] = (TL)(A12[irow * A.R.a12_rs + col] + dtt * v);
            }
        }
        __syncthreads();
    }
    if (FACC)
        for (int idx = tid; idx < NP * NP; idx += NTH) {
            const int i = idx / NP, c = idx - i * NP;
            const TA v = Acc[idx];
            if (v != (TA)0) A11[(a * NP + i) * A.R.a11_rs + b * NP + c] += (double)v;
        }
}

// ----------------------------------------------------------------------------
// A2 (FP64 form) by sum factorisation.  The volume contraction
//   Out[i][c] = sum_k sum_g dphi_k[g][i] G_k[g][c]
// (i a test function, c a block column, g a quadrature point, k a direction)
// has a tensor-product operator dphi_k = T_{k,0} (x) T_{k,1} (x) T_{k,2} with
// T_{k,r} the 1-D derivative table on axis r = k and the 1-D basis table
// elsewhere ((p+2) x (p+1) each).  It is applied one axis at a time to every
// column of G_k: (p+2)^2 (p+1) + (p+2)(p+1)^2 + (p+1)^3 multiply-adds per
// column and direction in 3-D instead of (p+1)^3 (p+2)^3.  G_k is generated
// from the point coefficients exactly as in k_blocks.  One CTA per (element,
// component pair), columns in chunks of CW; the face terms follow in
// k_blocks<..., VOL = false>.
// ----------------------------------------------------------------------------
template <class C, class TA = double>
struct SfShape {
    static constexpr int N1 = C::P + 1, Q1 = C::P + 2;
    static constexpr int NCB = C::NP + C::NF * C::NFP;
    // columns per chunk: 16 in FP64 (the FP64 pipe bounds the kernel), 32 in FP32, where the
    // per-chunk barriers and coefficient reloads, not the FMAs, set the time
    static constexpr int CW = sizeof(TA) == 4 ? 32 : 16;
    static constexpr int NX = (C::D == 3) ? Q1 * Q1 * N1 : Q1 * N1;      // after the first axis
    static constexpr int NY = (C::D == 3) ? Q1 * N1 * N1 : 0;            // after the second (3-D)
    static constexpr int NTH = 128;
    static constexpr int SLOTS = (C::NP * CW + NTH - 1) / NTH;
    static constexpr int smem_words = C::NCOEF * C::NQ + CW * (C::NQ + NX + NY);   // in the accumulation type
};

template <class C, class TA, class TL>
__global__ void __launch_bounds__(SfShape<C, TA>::NTH) k_blocks_sf(BlkArgs<TL> A) {
    using S = SfShape<C, TA>;
    constexpr int D = C::D, M = C::M, NP = C::NP, NQ = C::NQ, NFP = C::NFP, NCOEF = C::NCOEF;
    constexpr int N1 = S::N1, Q1 = S::Q1, NCB = S::NCB, CW = S::CW, NTH = S::NTH;
    constexpr int GEO = Geo<D>::N;
    const int tid = threadIdx.x;
    const int64_t bid = blockIdx.x;
    const int b = (int)(bid % M), a = (int)((bid / M) % M);
    const int64_t el = bid / (M * M), e = A.e0 + el;
    const DeviceTables& T = A.tab;
    // tables in the accumulation type (FP64 form: double; mixed form: float)
    constexpr bool F32 = sizeof(TA) == 4;
    const TA* tphi = F32 ? (const TA*)T.fphi : (const TA*)T.phi;
    const TA* tpsi = F32 ? (const TA*)T.fpsi : (const TA*)T.psi;
    const TA* ttheta = F32 ? (const TA*)T.ftheta : (const TA*)T.theta;
    const TA* tb1 = F32 ? (const TA*)T.fb1 : (const TA*)T.b1;
    const TA* td1 = F32 ? (const TA*)T.fd1 : (const TA*)T.d1;
    extern __shared__ double sm_raw[];
    TA* cs = reinterpret_cast<TA*>(sm_raw);   // [NCOEF][Nq] coefficients of one direction
    TA* Gs = cs + NCOEF * NQ;        // [Nq][CW]
    TA* Xs = Gs + NQ * CW;           // [NX][CW]
    TA* Ys = Xs + S::NX * CW;        // [NY][CW] (3-D)
    const TA* cf = static_cast<const TA*>(A.vcoef) + (((size_t)el * M + a) * M + b) * (size_t)(D * NCOEF * NQ);
    const double detJ = A.geo[e * GEO];
    double* A11 = A.R.a11 + e * A.R.a11_es;
    TL* A12 = A.R.a12 + e * A.R.a12_es;
#pragma unroll 1
    for (int c0 = 0; c0 < NCB; c0 += CW) {
        const int cw = min(CW, NCB - c0);
        TA acc[S::SLOTS];
#pragma unroll
        for (int s = 0; s < S::SLOTS; ++s) acc[s] = (TA)0;
#pragma unroll 1
        for (int k = 0; k < D; ++k) {
            __syncthreads();                 // the previous direction is done with cs / Gs
            for (int idx = tid; idx < NCOEF * NQ; idx += NTH) cs[idx] = cf[(size_t)k * NCOEF * NQ + idx];
            __syncthreads();
            for (int idx = tid; idx < NQ * CW; idx += NTH) {
                const int g = idx / CW, cc = idx - g * CW, c = c0 + cc;
                TA v = (TA)0;
                if (cc < cw) {
                    if (c < NP) {
                        v = cs[g] * tphi[g * NP + c];
                        for (int r2 = 0; r2 < D; ++r2) v -= cs[(1 + r2) * NQ + g] * tpsi[((size_t)r2 * NQ + g) * NP + c];
                    } else {
                        const int c2 = c - NP, f = c2 / NFP, l = c2 - f * NFP;
                        v = cs[(1 + D + f) * NQ + g] * ttheta[((size_t)f * NQ + g) * NFP + l];
                    }
                }
                Gs[idx] = v;
            }
            __syncthreads();
            const TA* T0 = (k == 0) ? td1 : tb1;
            const TA* T1 = (k == 1) ? td1 : tb1;
            if (D == 3) {
                const TA* T2 = (k == 2) ? td1 : tb1;
                // X[j2][g1][g0] = sum_g2 T2[g2][j2] G[g0 + Q1 g1 + Q1^2 g2]
                for (int idx = tid; idx < S::NX * CW; idx += NTH) {
                    const int cc = idx % CW, rest = idx / CW, j2 = rest % N1, g01 = rest / N1;
                    TA s = (TA)0;
#pragma unroll
                    for (int g2 = 0; g2 < Q1; ++g2) s = fma(T2[g2 * N1 + j2], Gs[(g01 + Q1 * Q1 * g2) * CW + cc], s);
                    Xs[(j2 * Q1 * Q1 + g01) * CW + cc] = s;
                }
                __syncthreads();
                // Y[j2][j1][g0] = sum_g1 T1[g1][j1] X[j2][g1][g0]
                for (int idx = tid; idx < S::NY * CW; idx += NTH) {
                    const int cc = idx % CW, rest = idx / CW, g0 = rest % Q1, j12 = rest / Q1;
                    const int j1 = j12 % N1, j2 = j12 / N1;
                    TA s = (TA)0;
#pragma unroll
                    for (int g1 = 0; g1 < Q1; ++g1) s = fma(T1[g1 * N1 + j1], Xs[(j2 * Q1 * Q1 + g1 * Q1 + g0) * CW + cc], s);
                    Ys[(j12 * Q1 + g0) * CW + cc] = s;
                }
                __syncthreads();
                // out[j0 + N1 j12] += sum_g0 T0[g0][j0] Y[j12][g0]
#pragma unroll
                for (int s = 0; s < S::SLOTS; ++s) {
                    const int idx = tid + NTH * s;
                    if (idx < NP * CW) {
                        const int cc = idx % CW, j = idx / CW, j0 = j % N1, j12 = j / N1;
                        TA t = (TA)0;
#pragma unroll
                        for (int g0 = 0; g0 < Q1; ++g0) t = fma(T0[g0 * N1 + j0], Ys[(j12 * Q1 + g0) * CW + cc], t);
                        acc[s] += t;
                    }
                }
            } else {
                // X[j1][g0] = sum_g1 T1[g1][j1] G[g0 + Q1 g1]
                for (int idx = tid; idx < S::NX * CW; idx += NTH) {
                    const int cc = idx % CW, rest = idx / CW, g0 = rest % Q1, j1 = rest / Q1;
                    TA s = (TA)0;
#pragma unroll
                    for (int g1 = 0; g1 < Q1; ++g1) s = fma(T1[g1 * N1 + j1], Gs[(g0 + Q1 * g1) * CW + cc], s);
                    Xs[(j1 * Q1 + g0) * CW + cc] = s;
                }
                __syncthreads();
#pragma unroll
                for (int s = 0; s < S::SLOTS; ++s) {
                    const int idx = tid + NTH * s;
                    if (idx < NP * CW) {
                        const int cc = idx % CW, j = idx / CW, j0 = j % N1, j1 = j / N1;
                        TA t = (TA)0;
#pragma unroll
                        for (int g0 = 0; g0 < Q1; ++g0) t = fma(T0[g0 * N1 + j0], Xs[(j1 * Q1 + g0) * CW + cc], t);
                        acc[s] += t;
                    }
                }
            }
        }
        // the chunk's columns of At (with the DIRK mass term) and Bt
#pragma unroll
        for (int s = 0; s < S::SLOTS; ++s) {
            const int idx = tid + NTH * s;
            if (idx >= NP * CW) continue;
            const int cc = idx % CW, i = idx / CW, c = c0 + cc;
            if (cc >= cw) continue;
            const int64_t row = a * NP + i;
            if (c < NP) {
                double v = (double)acc[s];
                if (a == b) v += detJ / A.a_ii * T.mhat[i * NP + c];
                A11[row * A.R.a11_rs + b * NP + c] = v;
            } else {
                const int c2 = c - NP, f = c2 / NFP, l = c2 - f * NFP;
                A12[row * A.R.a12_rs + (f * M + b) * NFP + l] = (TL)acc[s];
            }
        }
    }
}

// ----------------------------------------------------------------------------
// A3 + A4: bordered Gaussian elimination (interior LU, solves and Schur complement)
// ----------------------------------------------------------------------------
// One 64 x 64 (or smaller, NII / NJJ groups of 16) tile of the trailing
// update A22 -= L21 U12: thread (tx, ty) owns rows rb + ty + 16 ii and
// columns ct + tx + 16 jj.
template <int NII, int NJJ, int NB, int NR, int NC, int TCW, class RowP>
__device__ __forceinline__ void trail_tile(RowP rowp, const double* pan, const double* ust, int rb, int ct, int k0,
                                           int kb, int tx, int ty) {
    double acc[NII][NJJ];
    double* rp[NII];
#pragma unroll
    for (int ii = 0; ii < NII; ++ii) {
        int r = rb + ty + 16 * ii;
        rp[ii] = (r < NR) ? rowp(r) : nullptr;
#pragma unroll
        for (int jj = 0; jj < NJJ; ++jj) {
            int c = ct + tx + 16 * jj;
            acc[ii][jj] = (rp[ii] && c < NC) ? rp[ii][c] : 0.0;
        }
    }
    const double* lp = pan + (size_t)(rb + ty - k0) * NB;
    for (int j = 0; j < kb; ++j) {
        double lv[NII], uv[NJJ];
#pragma unroll
        for (int ii = 0; ii < NII; ++ii) lv[ii] = (rb + ty + 16 * ii < NR) ? lp[16 * ii * NB + j] : 0.0;
#pragma unroll
        for (int jj = 0; jj < NJJ; ++jj) uv[jj] = ust[j * TCW + tx + 16 * jj];
#pragma unroll
        for (int ii = 0; ii < NII; ++ii)
#pragma unroll
            for (int jj = 0; jj < NJJ; ++jj) acc[ii][jj] = fma(-lv[ii], uv[jj], acc[ii][jj]);
    }
#pragma unroll
    for (int ii = 0; ii < NII; ++ii) {
        if (!rp[ii]) continue;
#pragma unroll
        for (int jj = 0; jj < NJJ; ++jj) {
            int c = ct + tx + 16 * jj;
            if (c < NC) rp[ii][c] = acc[ii][jj];
        }
    }
}

template <class C, int NB>
constexpr int elim_smem_doubles() { return C::NR * NB + NB * 64; }

// Bordered elimination of one element.  NOSCHUR: the trace rows' trace columns
// (Dt) are left untouched, so that afterwards the trace rows hold the
// multipliers W = Ct U^{-1} in their interior columns and the right-hand side
// Rh - W z in their last column, and the interior rows hold Z = L^{-1} P Bt in
// their trace columns; the Schur product S = Dt - W Z is then formed by
// k_schur_ozaki on the tensor cores.
template <class C, int NB, int NTH, int MINB, bool NOSCHUR = false>
__global__ void __launch_bounds__(NTH, MINB) k_elim(double* top, double* bot, int64_t e0, int32_t* status) {
    constexpr int NU = C::NU, NR = C::NR, NC = C::NC, LD = C::LD;
    constexpr int TCW = 64;                 // column tile of the trailing update
    static_assert(NTH == 256, "trailing-update layout assumes 256 threads");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t el = blockIdx.x, e = e0 + el;
    double* Tm = top + e * (size_t)NU * LD;
    double* Bm = bot + el * (size_t)(NR - NU) * LD;
    auto rowp = [&](int r) -> double* { return r < NU ? Tm + (size_t)r * LD : Bm + (size_t)(r - NU) * LD; };
    extern __shared__ double sm[];
    double* pan = sm;                       // [NR][NB], row index relative to k0
    double* ust = pan + NR * NB;            // [NB][TCW]
    __shared__ int piv[NB];
    __shared__ int sflag;
    if (tid == 0) sflag = 0;

    for (int k0 = 0; k0 < NU; k0 += NB) {
        const int kb = min(NB, NU - k0), nrows = NR - k0, ntop = NU - k0;
#pragma unroll 1
        for (int idx = tid; idx < nrows * kb; idx += NTH) {
            int rr = idx / kb, c = idx - rr * kb;
            pan[rr * NB + c] = rowp(k0 + rr)[k0 + c];
        }
        __syncthreads();
        for (int j = 0; j < kb; ++j) {
            // warp 0 alone: pivot search (largest magnitude, lowest row on ties) and the row
            // interchange inside the panel; one barrier per step
            if (warp == 0) {
                double bv = -1.0;
                int bi = INT_MAX;
#pragma unroll 1
                for (int rr = j + lane; rr < ntop; rr += 32) {
                    const double v = fabs(pan[rr * NB + j]);
                    if (v > bv) { bv = v; bi = rr; }
                }
                for (int off = 16; off > 0; off >>= 1) {
                    const double ov = __shfl_down_sync(0xffffffffu, bv, off);
                    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
                    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
                }
                int pr = __shfl_sync(0xffffffffu, bi, 0);
                if (pr == INT_MAX) {
                    pr = j;
                    if (lane == 0) sflag |= 2;
                }
                if (lane < kb && pr != j) {
                    const double t = pan[j * NB + lane];
                    pan[j * NB + lane] = pan[pr * NB + lane];
                    pan[pr * NB + lane] = t;
                }
                if (lane == 0) piv[j] = pr;
            }
            __syncthreads();
            double pv = pan[j * NB + j];
            if (pv == 0.0 || !isfinite(pv)) {
                if (tid == 0) sflag |= (pv == 0.0) ? 1 : 2;
                pv = 1.0;
            }
            const double inv = 1.0 / pv;
#pragma unroll 1
            for (int rr = j + 1 + tid; rr < nrows; rr += NTH) {
                double l = pan[rr * NB + j] * inv;
                pan[rr * NB + j] = l;
                for (int c = j + 1; c < kb; ++c) pan[rr * NB + c] = fma(-l, pan[j * NB + c], pan[rr * NB + c]);
            }
            __syncthreads();
        }
#pragma unroll 1
        for (int idx = tid; idx < nrows * kb; idx += NTH) {
            int rr = idx / kb, c = idx - rr * kb;
            rowp(k0 + rr)[k0 + c] = pan[rr * NB + c];
        }
        // trailing columns: row swaps and U12 = L11^{-1} A12 (each thread owns columns)
        const int c0 = k0 + kb;
#pragma unroll 1
        for (int c = c0 + tid; c < NC; c += NTH) {
            for (int j = 0; j < kb; ++j) {
                int pr = piv[j];
                if (pr != j) {
                    double* x = rowp(k0 + j) + c;
                    double* y = rowp(k0 + pr) + c;
                    double t = *x; *x = *y; *y = t;
                }
            }
            double xv[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                if (j < kb) {
                    double s = rowp(k0 + j)[c];
#pragma unroll
                    for (int i = 0; i < NB; ++i)
                        if (i < j) s = fma(-pan[j * NB + i], xv[i], s);
                    xv[j] = s;
                    rowp(k0 + j)[c] = s;
                }
            }
        }
        __syncthreads();
        // trailing update A22 -= L21 U12 on rows [c0, NR) x cols [c0, NC)
        const int tx = tid & 15, ty = tid >> 4;
        if constexpr (NOSCHUR) {
            // interior rows: all trailing columns; trace rows: interior columns and the
            // right-hand side only (the trace-trace block waits for the Schur product)
#pragma unroll 1
            for (int ct = c0; ct < NC; ct += TCW) {
                for (int idx = tid; idx < kb * TCW; idx += NTH) {
                    int j = idx / TCW, cc = idx - j * TCW;
                    ust[j * TCW + cc] = (ct + cc < NC) ? rowp(k0 + j)[ct + cc] : 0.0;
                }
                __syncthreads();
                int njj = 0;
                while (njj < 4 && ct + 16 * njj < NC) ++njj;
#pragma unroll 1
                for (int rb = c0; rb < NU; rb += 64) {
                    int nii = 0;
                    while (nii < 4 && rb + 16 * nii < NU) ++nii;
                    switch (nii * 4 + njj - 5) {
#define HDG_TT(I, J) case (I) * 4 + (J) - 5: trail_tile<I, J, NB, NU, NC, TCW>(rowp, pan, ust, rb, ct, k0, kb, tx, ty); break;
                        HDG_TT(1, 1) HDG_TT(1, 2) HDG_TT(1, 3) HDG_TT(1, 4)
                        HDG_TT(2, 1) HDG_TT(2, 2) HDG_TT(2, 3) HDG_TT(2, 4)
                        HDG_TT(3, 1) HDG_TT(3, 2) HDG_TT(3, 3) HDG_TT(3, 4)
                        HDG_TT(4, 1) HDG_TT(4, 2) HDG_TT(4, 3) HDG_TT(4, 4)
#undef HDG_TT
                        default: break;
                    }
                }
                if (ct < NU) {
                    int njt = 0;
                    while (njt < 4 && ct + 16 * njt < NU) ++njt;
#pragma unroll 1
                    for (int rb = NU; rb < NR; rb += 64) {
                        int nii = 0;
                        while (nii < 4 && rb + 16 * nii < NR) ++nii;
                        switch (nii * 4 + njt - 5) {
#define HDG_TT(I, J) case (I) * 4 + (J) - 5: trail_tile<I, J, NB, NR, NU, TCW>(rowp, pan, ust, rb, ct, k0, kb, tx, ty); break;
                            HDG_TT(1, 1) HDG_TT(1, 2) HDG_TT(1, 3) HDG_TT(1, 4)
                            HDG_TT(2, 1) HDG_TT(2, 2) HDG_TT(2, 3) HDG_TT(2, 4)
                            HDG_TT(3, 1) HDG_TT(3, 2) HDG_TT(3, 3) HDG_TT(3, 4)
                            HDG_TT(4, 1) HDG_TT(4, 2) HDG_TT(4, 3) HDG_TT(4, 4)
#undef HDG_TT
                            default: break;
                        }
                    }
                }
                __syncthreads();
            }
#pragma unroll 1
            for (int r = NU + tid; r < NR; r += NTH) {       // right-hand side of the trace rows
                double s = rowp(r)[NC - 1];
                for (int j = 0; j < kb; ++j) s = fma(-pan[(r - k0) * NB + j], rowp(k0 + j)[NC - 1], s);
                rowp(r)[NC - 1] = s;
            }
            __syncthreads();
        } else {
#pragma unroll 1
        for (int ct = c0; ct < NC; ct += TCW) {
            for (int idx = tid; idx < kb * TCW; idx += NTH) {
                int j = idx / TCW, cc = idx - j * TCW;
                ust[j * TCW + cc] = (ct + cc < NC) ? rowp(k0 + j)[ct + cc] : 0.0;
            }
            __syncthreads();
            int njj = 0;                       // column groups of 16 inside the matrix (warp-uniform)
            while (njj < 4 && ct + 16 * njj < NC) ++njj;
#pragma unroll 1
            for (int rb = c0; rb < NR; rb += 64) {
                int nii = 0;                   // row groups of 16 inside the matrix (warp-uniform)
                while (nii < 4 && rb + 16 * nii < NR) ++nii;
                switch (nii * 4 + njj - 5) {
#define HDG_TT(I, J) case (I) * 4 + (J) - 5: trail_tile<I, J, NB, NR, NC, TCW>(rowp, pan, ust, rb, ct, k0, kb, tx, ty); break;
                    HDG_TT(1, 1) HDG_TT(1, 2) HDG_TT(1, 3) HDG_TT(1, 4)
                    HDG_TT(2, 1) HDG_TT(2, 2) HDG_TT(2, 3) HDG_TT(2, 4)
                    HDG_TT(3, 1) HDG_TT(3, 2) HDG_TT(3, 3) HDG_TT(3, 4)
                    HDG_TT(4, 1) HDG_TT(4, 2) HDG_TT(4, 3) HDG_TT(4, 4)
#undef HDG_TT
                    default: break;
                }
            }
            __syncthreads();
        }
        }
    }
    if (tid == 0 && sflag) atomicOr(status, sflag);
}

// ----------------------------------------------------------------------------
// A5: deterministic assembly of S^K and g^K into the block-sparse trace system
// ----------------------------------------------------------------------------
template <class C>
__global__ void k_assemble(const double* bot, int64_t e0, const int32_t* blk, const int32_t* rank,
                           const int32_t* iperm, double* vals, int pass) {
    constexpr int M = C::M, NF = C::NF, NFP = C::NFP, NU = C::NU, NT = C::NT, LD = C::LD, BS = C::BS;
    const int64_t bid = blockIdx.x;
    const int gl = (int)(bid % NF), fl = (int)((bid / NF) % NF);
    const int64_t el = bid / (NF * NF), e = e0 + el;
    const size_t item = ((size_t)e * NF + fl) * NF + gl;
    if (rank[item] != pass) return;
    double* out = vals + (size_t)blk[item] * BS * BS;
    const double* Bm = bot + el * (size_t)NT * LD;
    const int32_t* ipf = iperm + ((size_t)e * NF + fl) * NFP;
    const int32_t* ipg = iperm + ((size_t)e * NF + gl) * NFP;
    for (int idx = threadIdx.x; idx < BS * BS; idx += blockDim.x) {
        int c = idx / BS, r = idx - c * BS;
        int a = r / NFP, k = r - a * NFP, b2 = c / NFP, k2 = c - b2 * NFP;
        int row = (fl * M + a) * NFP + ipf[k];
        int col = NU + (gl * M + b2) * NFP + ipg[k2];
        out[idx] += Bm[(size_t)row * LD + col];
    }
}

template <class C>
__global__ void k_assemble_g(const double* bot, int64_t e0, const int32_t* e2f, const int32_t* frank,
                             const int32_t* iperm, double* g, int pass) {
    constexpr int M = C::M, NF = C::NF, NFP = C::NFP, NT = C::NT, LD = C::LD, NC = C::NC, BS = C::BS;
    const int64_t bid = blockIdx.x;
    const int fl = (int)(bid % NF);
    const int64_t el = bid / NF, e = e0 + el;
    if (frank[e * NF + fl] != pass) return;
    const int64_t F = e2f[e * NF + fl];
    const double* Bm = bot + el * (size_t)NT * LD;
    const int32_t* ipf = iperm + ((size_t)e * NF + fl) * NFP;
    for (int idx = threadIdx.x; idx < BS; idx += blockDim.x) {
        int a = idx / NFP, k = idx - a * NFP;
        int row = (fl * M + a) * NFP + ipf[k];
        g[F * BS + idx] -= Bm[(size_t)row * LD + NC - 1];
    }
}

// ----------------------------------------------------------------------------
// A6: trace matvec y = S x (block rows, column-major blocks)
// ----------------------------------------------------------------------------
template <class C>
struct MvShape {
    static constexpr int RB = ((C::BS + 31) / 32) * 32;
    static constexpr int GROUPS = (RB <= 64) ? 4 : 2;
    static constexpr int NTH = RB * GROUPS;
};

template <class C>
__global__ void __launch_bounds__(MvShape<C>::NTH) k_matvec(const int32_t* rowptr, const int32_t* col,
                                                            const double* vals, const double* x, double* y) {
    constexpr int BS = C::BS, RB = MvShape<C>::RB, GROUPS = MvShape<C>::GROUPS;
    __shared__ double part[GROUPS][RB];
    const int64_t F = blockIdx.x;
    const int grp = threadIdx.x / RB, r = threadIdx.x - grp * RB;
    double acc0 = 0.0, acc1 = 0.0;
    if (r < BS) {
        for (int b = rowptr[F] + grp; b < rowptr[F + 1]; b += GROUPS) {
            const double* xs = x + (size_t)col[b] * BS;
            const double* v = vals + (size_t)b * BS * BS + r;
            int c = 0;
#pragma unroll 4
            for (; c + 1 < BS; c += 2) {
                acc0 = fma(v[(size_t)c * BS], xs[c], acc0);
                acc1 = fma(v[(size_t)(c + 1) * BS], xs[c + 1], acc1);
            }
            if (c < BS) acc0 = fma(v[(size_t)c * BS], xs[c], acc0);
        }
    }
    part[grp][r] = acc0 + acc1;
    __syncthreads();
    if (grp == 0 && r < BS) {
        double s = part[0][r];
        for (int g2 = 1; g2 < GROUPS; ++g2) s += part[g2][r];
        y[F * BS + r] = s;
    }
}

// ----------------------------------------------------------------------------
// A7: interior recovery dU = -U^{-1}(z + Z dUhat_K), dQ = dq0 - L dU + Lambda dUhat_K
// ----------------------------------------------------------------------------
// x = U^{-1} w for an upper-triangular, row-major FP64 matrix U in global
// memory (row stride ld, n rows), w and x in shared memory, by the whole CTA of
// NT threads: 32-row diagonal blocks from the bottom; the rows of a block are
// first reduced by the solved part (one warp per row, lanes along the row, so
// the reads are coalesced and a whole block's rows are in flight at once), the
// block's 32 x 32 diagonal part is staged in shared memory, and warp 0 solves
// it with shuffles.  The serial chain is n / 32 block steps instead of n
// dependent row reads.  sD: 32 x 33 doubles, part: 32 doubles of shared memory.
template <int NT>
__device__ void upper_solve_blocked(const double* U, int64_t ld, int n, const double* w, double* x, double* sD,
                                    double* part) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = NT / 32;
#pragma unroll 1
    for (int b1 = n; b1 > 0; b1 -= 32) {
        const int b0 = max(0, b1 - 32), nb = b1 - b0;
        for (int rr = warp; rr < nb; rr += NW) {
            const double* row = U + (int64_t)(b0 + rr) * ld;
            double s = 0.0;
            for (int j = b1 + lane; j < n; j += 32) s = fma(row[j], x[j], s);
            for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
            if (lane == 0) part[rr] = s;
        }
        for (int idx = tid; idx < nb * 32; idx += NT) {
            const int r = idx >> 5, c = idx & 31;
            if (c < nb) sD[r * 33 + c] = U[(int64_t)(b0 + r) * ld + b0 + c];
        }
        __syncthreads();
        if (warp == 0) {
            double v = lane < nb ? w[b0 + lane] - part[lane] : 0.0;
            for (int k = nb - 1; k >= 0; --k) {
                if (lane == k) v = v / sD[k * 33 + k];
                const double xk = __shfl_sync(0xffffffffu, v, k);
                if (lane < k) v = fma(-sD[lane * 33 + k], xk, v);
            }
            if (lane < nb) x[b0 + lane] = v;
        }
        __syncthreads();
    }
}

struct RecArgs {
    const double* top; const double* dq0; const double* geo;
    DeviceTables tab;
    const int32_t* e2f; const int32_t* perm;
    const double* dUH; double* dQ; double* dU;
};

template <class C, int NTH>
__global__ void __launch_bounds__(NTH) k_recover(RecArgs A) {
    constexpr int D = C::D, M = C::M, NP = C::NP, NF = C::NF, NFP = C::NFP;
    constexpr int NU = C::NU, NQV = C::NQV, NT = C::NT, LD = C::LD, NC = C::NC;
    constexpr int GEO = Geo<D>::N;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t e = blockIdx.x;
    __shared__ double duh[NT];
    __shared__ double w[NU];
    __shared__ double x[NU];
    __shared__ double geo[GEO];
    __shared__ double sD[32 * 33];
    __shared__ double part[32];
    for (int i = tid; i < NT; i += NTH) {
        int f = i / (M * NFP), rem = i - f * M * NFP, a = rem / NFP, l = rem - a * NFP;
        int64_t F = A.e2f[e * NF + f];
        int k = A.perm[(e * NF + f) * NFP + l];
        duh[i] = A.dUH[(F * M + a) * NFP + k];
    }
    for (int i = tid; i < GEO; i += NTH) geo[i] = A.geo[e * GEO + i];
    __syncthreads();
    const double* Tm = A.top + e * (size_t)NU * LD;
    for (int i = warp; i < NU; i += NTH / 32) {
        const double* row = Tm + (size_t)i * LD;
        double s = 0.0;
#pragma unroll
        for (int c = lane; c < NT; c += 32) s = fma(row[NU + c], duh[c], s);
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) w[i] = s + row[NC - 1];
    }
    __syncthreads();
    upper_solve_blocked<NTH>(Tm, LD, NU, w, x, sD, part);
    for (int i = tid; i < NU; i += NTH) A.dU[e * NU + i] = -x[i];
    const double detJ = geo[0];
    const double* Jinv = geo + 1;
    const double* NW = geo + 1 + D * D;
    const DeviceTables& T = A.tab;
    for (int idx = tid; idx < M * NP; idx += NTH) {
        int b = idx / NP, i = idx - b * NP;
        double t[D], ef[NF];
        for (int r = 0; r < D; ++r) {
            double s = 0.0;
            const double* mc = T.minv_c + ((size_t)r * NP + i) * NP;
            for (int j = 0; j < NP; ++j) s -= mc[j] * x[b * NP + j];   // dU = -x
            t[r] = s;
        }
        for (int f = 0; f < NF; ++f) {
            double s = 0.0;
            const double* me = T.minv_e + ((size_t)f * NP + i) * NFP;
            for (int l = 0; l < NFP; ++l) s += me[l] * duh[(f * M + b) * NFP + l];
            ef[f] = s;
        }
        for (int l = 0; l < D; ++l) {
            double v = 0.0;
            for (int r = 0; r < D; ++r) v -= Jinv[r * D + l] * t[r];
            for (int f = 0; f < NF; ++f) v += NW[f * D + l] / detJ * ef[f];
            int o = (l * M + b) * NP + i;
            A.dQ[e * NQV + o] = A.dq0[e * NQV + o] + v;
        }
    }
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
template <class C> struct BlkCfg;
template <> struct BlkCfg<Cfg<2, 1>> { static constexpr int TY = 4, TX = 8, KC = 16; };
template <> struct BlkCfg<Cfg<2, 2>> { static constexpr int TY = 4, TX = 8, KC = 16; };
template <> struct BlkCfg<Cfg<2, 3>> { static constexpr int TY = 8, TX = 8, KC = 16; };
template <> struct BlkCfg<Cfg<3, 1>> { static constexpr int TY = 8, TX = 8, KC = 16; };
template <> struct BlkCfg<Cfg<3, 2>> { static constexpr int TY = 8, TX = 16, KC = 16; };
template <> struct BlkCfg<Cfg<3, 3>> { static constexpr int TY = 16, TX = 16, KC = 16; };

#define HDG_CK(call)                                                                   \
    do {                                                                               \
        cudaError_t err_ = (call);                                                     \
        if (err_ != cudaSuccess) {                                                     \
            h->err = std::string(#call) + ": " + cudaGetErrorString(err_);             \
            return HDG_ECUDA;                                                          \
        }                                                                              \
    } while (0)

// Element Schur complements S^K to the caller's buffer (hdg_set_element_block_output):
// out[e][r][c] = the element's trace-trace block after condensation, rows and columns
// in the element's local trace order (local face, component, local face node); one
// CTA per element of the chunk, src row stride rs, first trace column col0.
template <class TS, class TO>
__global__ void k_copy_sk(const TS* src, int64_t src_es, int64_t rs, int64_t col0, int nt, int64_t e0, TO* out) {
    const int64_t el = blockIdx.x;
    const TS* S = src + el * src_es + col0;
    TO* o = out + (e0 + el) * (int64_t)nt * nt;
    for (int idx = threadIdx.x; idx < nt * nt; idx += blockDim.x) {
        const int r = idx / nt, c = idx - r * nt;
        o[idx] = (TO)S[(int64_t)r * rs + c];
    }
}

}  // namespace hdg

// FP64 Schur product on the tensor cores (defined before its launch below)
#include "ozaki.cuh"

namespace hdg {

template <int D, int P>
int run_linearize(hdg_ctx* h, const LinArgs& la) {
    if (int rc = ensure_system_storage(h, HDG_PREC_FP64)) return rc;
    using C = Cfg<D, P>;
    using BC = BlkCfg<C>;
    using BS_ = BlkShape<C, BC::TY, BC::TX, BC::KC>;
    auto kblk = k_blocks<C, BC::TY, BC::TX, BC::KC, double, double>;
    auto kface = k_blocks<C, BC::TY, BC::TX, BC::KC, double, double, false>;
    constexpr int PT = 128;
    const size_t sm_sf = sizeof(double) * SfShape<C>::smem_words;
    const size_t sm_point = sizeof(double) * point_smem_doubles<C>();
    const size_t sm_blk = sizeof(double) * BS_::smem;
    const size_t sm_elim16 = sizeof(double) * elim_smem_doubles<C, 16>();
    const size_t sm_elim8 = sizeof(double) * elim_smem_doubles<C, 8>();
    HDG_CK(cudaFuncSetAttribute(k_point<C, PT, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_point));
    HDG_CK(cudaFuncSetAttribute(kblk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_blk));
    HDG_CK(cudaFuncSetAttribute(kface, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_blk));
    HDG_CK(cudaFuncSetAttribute(k_blocks_sf<C, double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_sf));
    HDG_CK(cudaFuncSetAttribute(k_elim<C, 16, 256, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_elim16));
    HDG_CK(cudaFuncSetAttribute(k_elim<C, 16, 256, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_elim16));
    HDG_CK(cudaFuncSetAttribute(k_elim<C, 8, 256, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_elim8));
    HDG_CK(cudaFuncSetAttribute(k_elim<C, 8, 256, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_elim8));
    const bool oz = h->schur64_mode == 1;   // Schur product emulated on the tensor cores
    if (oz) {
        HDG_CK(cudaFuncSetAttribute(k_elim<C, 16, 256, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_elim16));
        HDG_CK(cudaFuncSetAttribute(k_elim<C, 16, 256, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_elim16));
        HDG_CK(cudaFuncSetAttribute(k_elim<C, 8, 256, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_elim8));
        HDG_CK(cudaFuncSetAttribute(k_elim<C, 8, 256, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_elim8));
        HDG_CK(cudaFuncSetAttribute(k_schur_ozaki<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, OzakiCfg<C>::SMEM));
    }
    cudaStream_t st = h->stream;
    HDG_CK(cudaMemsetAsync(h->d_vals, 0, sizeof(double) * h->nnzb * C::BS * C::BS, st));
    HDG_CK(cudaMemsetAsync(h->d_g, 0, sizeof(double) * h->F * C::BS, st));
    PointArgs pa;
    pa.U = la.U; pa.Q = la.Q; pa.UH = la.UH; pa.Ustar = la.Ustar; pa.nu = la.nu;
    pa.dt = la.dt; pa.a_ii = la.a_ii; pa.ph = phys_t<double>(h->phys); pa.phf = phys_t<float>(h->phys);
    pa.tau = h->phys.tau; pa.tab = h->tab; pa.geo = h->d_geo;
    const Regions<double> RG = fp64_regions<C>(h->d_top, h->d_bot);
    pa.e2f = h->d_e2f; pa.perm = h->d_perm;
    pa.rt = RG.rt; pa.rt_es = RG.rt_es; pa.rt_rs = RG.rt_rs;
    pa.rb = RG.rb; pa.rb_es = RG.rb_es; pa.rb_rs = RG.rb_rs;
    pa.vcoef = h->d_vcoef; pa.fcoef = h->d_fcoef; pa.dq0 = h->d_dq0;
    pa.ftag = h->d_ftag; pa.ub = h->d_ub; pa.ubf = h->d_ubf; pa.ew = h->e_wall;
    pa.tau_mode = h->phys.tau_mode; pa.taup = h->phys.tau_mode ? h->d_taup : nullptr;
    BlkArgs<double> ba;
    ba.vcoef = h->d_vcoef; ba.fcoef = h->d_fcoef; ba.geo = h->d_geo; ba.tab = h->tab; ba.ftag = h->d_ftag;
    ba.ew = h->e_wall;
    ba.taup = h->phys.tau_mode ? h->d_taup : nullptr;
    ba.R = RG; ba.dt = la.dt; ba.a_ii = la.a_ii; ba.tau = h->phys.tau;
    for (int64_t e0 = 0; e0 < h->E; e0 += h->chunk) {
        const int64_t ne = std::min<int64_t>(h->chunk, h->E - e0);
        pa.e0 = e0; ba.e0 = e0;
        prof_begin(h, HDG_K_POINT);
        k_point<C, PT, double><<<(unsigned)ne, PT, sm_point, st>>>(pa);
        prof_end(h);
        prof_begin(h, HDG_K_BLOCKS);
        if (h->blocks64_mode == 1) {         // sum-factorised volume terms, then the face terms
            k_blocks_sf<C, double, double><<<(unsigned)(ne * C::M * C::M), SfShape<C>::NTH, sm_sf, st>>>(ba);
            kface<<<(unsigned)(ne * C::M * C::M), BC::TY * BC::TX, sm_blk, st>>>(ba);
        } else {
            kblk<<<(unsigned)(ne * C::M * C::M), BC::TY * BC::TX, sm_blk, st>>>(ba);
        }
        prof_end(h);
        prof_begin(h, HDG_K_ELIM);
        // variant chosen by the autotuner: panel width 16 or 8, built for 1 or 2 resident CTAs per SM
        if (oz) {
            if (h->elim_nb == 8) {
                if (h->elim_minb == 1)
                    k_elim<C, 8, 256, 1, true><<<(unsigned)ne, 256, sm_elim8, st>>>(h->d_top, h->d_bot, e0, h->d_status);
                else
                    k_elim<C, 8, 256, 2, true><<<(unsigned)ne, 256, sm_elim8, st>>>(h->d_top, h->d_bot, e0, h->d_status);
            } else {
                if (h->elim_minb == 1)
                    k_elim<C, 16, 256, 1, true><<<(unsigned)ne, 256, sm_elim16, st>>>(h->d_top, h->d_bot, e0, h->d_status);
                else
                    k_elim<C, 16, 256, 2, true><<<(unsigned)ne, 256, sm_elim16, st>>>(h->d_top, h->d_bot, e0, h->d_status);
            }
            prof_end(h);
            prof_begin(h, HDG_K_SCHUR);
            k_oz_scales<C><<<(unsigned)ne, 256, 0, st>>>(h->d_top, h->d_bot, e0, h->d_ozexp);
            CUtensorMap tmW, tmZ;                 // trace rows of this chunk, interior rows of every element
            std::string terr;
            if (make_tmap_f64_3d(&tmW, h->d_bot, C::LD, C::NT, (uint64_t)ne, 8ull * C::LD, 8ull * C::LD * C::NT,
                                 OzakiCfg<C>::WRS, OzakiCfg<C>::MT, terr) ||
                make_tmap_f64_3d(&tmZ, h->d_top, C::LD, C::NU, (uint64_t)h->E, 8ull * C::LD, 8ull * C::LD * C::NU,
                                 OzakiCfg<C>::ZRS, OzakiCfg<C>::KC, terr)) {
                h->err = terr;
                return HDG_ECUDA;
            }
            k_schur_ozaki<C><<<(unsigned)(ne * OzakiCfg<C>::NMT * OzakiCfg<C>::NNT), OZ_THREADS, OzakiCfg<C>::SMEM, st>>>(
                h->d_top, h->d_bot, e0, h->d_ozexp, h->d_status, tmW, tmZ);
        } else if (h->elim_nb == 8) {
            if (h->elim_minb == 1)
                k_elim<C, 8, 256, 1><<<(unsigned)ne, 256, sm_elim8, st>>>(h->d_top, h->d_bot, e0, h->d_status);
            else
                k_elim<C, 8, 256, 2><<<(unsigned)ne, 256, sm_elim8, st>>>(h->d_top, h->d_bot, e0, h->d_status);
        } else {
            if (h->elim_minb == 1)
                k_elim<C, 16, 256, 1><<<(unsigned)ne, 256, sm_elim16, st>>>(h->d_top, h->d_bot, e0, h->d_status);
            else
                k_elim<C, 16, 256, 2><<<(unsigned)ne, 256, sm_elim16, st>>>(h->d_top, h->d_bot, e0, h->d_status);
        }
        prof_end(h);
        if (h->d_skout)
            k_copy_sk<double, double><<<(unsigned)ne, 256, 0, st>>>(h->d_bot, (int64_t)C::NT * C::LD, C::LD, C::NU,
                                                                    C::NT, e0, static_cast<double*>(h->d_skout));
        for (int pass = 0; pass < 2; ++pass) {
            prof_begin(h, HDG_K_ASSEMBLE);
            k_assemble<C><<<(unsigned)(ne * C::NF * C::NF), 256, 0, st>>>(h->d_bot, e0, h->d_blk, h->d_rank,
                                                                          h->d_iperm, h->d_vals, pass);
            prof_end(h);
            prof_begin(h, HDG_K_ASSEMBLE);
            k_assemble_g<C><<<(unsigned)(ne * C::NF), 128, 0, st>>>(h->d_bot, e0, h->d_e2f, h->d_frank,
                                                                   h->d_iperm, h->d_g, pass);
            prof_end(h);
        }
        HDG_CK(cudaGetLastError());
    }
    h->have_system = true;
    h->sys_prec = HDG_PREC_FP64;
    h->bj_ready = false;
    h->asm_ready = false;
    return HDG_OK;
}

template <int D, int P>
int run_matvec(hdg_ctx* h, const double* x, double* y);
template <int D, int P>
int run_recover_mixed(hdg_ctx* h, const double* dUH, double* dQ, double* dU);

template <int D, int P>
int run_recover(hdg_ctx* h, const double* dUH, double* dQ, double* dU) {
    using C = Cfg<D, P>;
    if (h->sys_prec == HDG_PREC_MIXED) return run_recover_mixed<D, P>(h, dUH, dQ, dU);
    RecArgs ra;
    ra.top = h->d_top; ra.dq0 = h->d_dq0; ra.geo = h->d_geo; ra.tab = h->tab;
    ra.e2f = h->d_e2f; ra.perm = h->d_perm; ra.dUH = dUH; ra.dQ = dQ; ra.dU = dU;
    prof_begin(h, HDG_K_RECOVER);
    k_recover<C, 256><<<(unsigned)h->E, 256, 0, h->stream>>>(ra);
    prof_end(h);
    HDG_CK(cudaGetLastError());
    return HDG_OK;
}

#define HDG_INSTANTIATE(D, P)                                                             \
    template int run_linearize<D, P>(hdg_ctx*, const LinArgs&);                           \
    template int run_matvec<D, P>(hdg_ctx*, const double*, double*);                      \
    template int run_recover<D, P>(hdg_ctx*, const double*, double*, double*);

}  // namespace hdg
