// Consumer side of the condensed system (FP64): the nonlinear stage residual
// F(W) = [R_q; R_u; R_uhat] (eq. nonlinear-residual), the Newton state update
// W <- W + alpha dW (eq. newton-update), a block-Jacobi preconditioner made of
// the inverses of the diagonal face blocks S_FF of the trace operator (the
// single-face special case of eq. additive-schwarz), and the vector kernels
// of restarted GMRES.
#pragma once

#include "mixed.cuh"
#include "schwarz.cuh"
#include "av.cuh"

namespace hdg {

// ----------------------------------------------------------------------------
// stage residual
// ----------------------------------------------------------------------------
struct ResArgs {
    const double* U; const double* Q; const double* UH; const double* Ustar; const double* nu;
    double dt, a_ii;
    PhysT<double> ph;
    double tau;
    int tau_mode;               // 0 constant tau, 1 state-dependent (stab_tau)
    DeviceTables tab;
    const double* geo;
    const int32_t* e2f; const int32_t* perm;
    double* Rq; double* Ru;      // optional outputs [E][d][m][Np], [E][m][Np]
    double* rk;                  // [E][nf][m][Nfp] element contributions to R_uhat
    double* part;                // [E] sum of squares of R_q and R_u of the element
    const int32_t* ftag;         // [E][nf] boundary tags or NULL
    const double* ub;            // [m] tag-1 boundary state
    const double* ubf;           // [F][m][Nfp] nodal tag-1 boundary data, or NULL
    double ew;                   // wall internal energy of tag-3 faces
};

// Lifted gradient at node i of component a (eq. hdg-grad with R_q = 0):
// Q_lift = M^{-1}(-C U + E Uhat), from the element's staged U and Uhat.
template <class C>
__device__ __forceinline__ void lift_at_node(const DeviceTables& T, const double* sU, const double* sUH,
                                             const double* Jinv, const double* NW, double detJ, int a, int i,
                                             double (&ql)[C::D]) {
    constexpr int D = C::D, M = C::M, NP = C::NP, NF = C::NF, NFP = C::NFP;
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
        double v = 0.0;
        for (int r = 0; r < D; ++r) v -= Jinv[r * D + l] * t[r];
        for (int f = 0; f < NF; ++f) v += NW[f * D + l] / detJ * ef[f];
        ql[l] = v;
    }
}

// Q = Q_lift(U, Uhat) for every element: the gradient for which R_q = 0
template <class C, int NTH>
__global__ void __launch_bounds__(NTH) k_lift(const double* __restrict__ U, const double* __restrict__ UH,
                                              double* __restrict__ Q, DeviceTables T, const double* __restrict__ geog,
                                              const int32_t* __restrict__ e2f, const int32_t* __restrict__ perm) {
    constexpr int D = C::D, M = C::M, NP = C::NP, NF = C::NF, NFP = C::NFP, NU = C::NU, NT = C::NT;
    constexpr int GEO = Geo<D>::N;
    __shared__ double sU[NU], sUH[NT], geo[GEO];
    const int tid = threadIdx.x;
    const int64_t e = blockIdx.x;
    for (int i = tid; i < NU; i += NTH) sU[i] = U[e * NU + i];
    for (int i = tid; i < NT; i += NTH) {
        int f = i / (M * NFP), rem = i - f * M * NFP, a = rem / NFP, l = rem - a * NFP;
        int64_t F = e2f[e * NF + f];
        sUH[i] = UH[(F * M + a) * NFP + perm[(e * NF + f) * NFP + l]];
    }
    for (int i = tid; i < GEO; i += NTH) geo[i] = geog[e * GEO + i];
    __syncthreads();
    for (int idx = tid; idx < M * NP; idx += NTH) {
        int a = idx / NP, i = idx - a * NP;
        double ql[D];
        lift_at_node<C>(T, sU, sUH, geo + 1, geo + 1 + D * D, geo[0], a, i, ql);
        for (int l = 0; l < D; ++l) Q[e * C::NQV + (l * M + a) * NP + i] = ql[l];
    }
}

template <class C>
constexpr int res_smem_doubles() {
    return C::NU + 2 * C::NQV + C::NP + 2 * C::NT + C::D * C::M * C::NQ + 2 * C::NF * C::M * C::NFQ + 32;
}

template <class C, int NTH>
__global__ void __launch_bounds__(NTH) k_residual(ResArgs A) {
    constexpr int D = C::D, M = C::M, NP = C::NP, NQ = C::NQ, NF = C::NF, NFP = C::NFP, NFQ = C::NFQ;
    constexpr int NU = C::NU, NQV = C::NQV, NT = C::NT;
    constexpr int GEO = Geo<D>::N;
    const int tid = threadIdx.x;
    const int64_t e = blockIdx.x;
    extern __shared__ double sm[];
    double* sU = sm;
    double* sQ = sU + NU;
    double* sQL = sQ + NQV;
    double* sNu = sQL + NQV;
    double* sUH = sNu + NP;
    double* sF = sUH + NT;               // [d][m][Nq]
    double* sFH = sF + D * M * NQ;       // [nf][m][Nfq]
    double* sRh = sFH + NF * M * NFQ;    // [nf][m][Nfp]
    double* sFB = sRh + NT;              // [nf][m][Nfq] bhat on boundary faces
    double* red = sFB + NF * M * NFQ;    // [32]
    __shared__ double geo[GEO];
    const DeviceTables& T = A.tab;
    for (int i = tid; i < NU; i += NTH) sU[i] = A.U[e * NU + i];
    for (int i = tid; i < NQV; i += NTH) sQ[i] = A.Q[e * NQV + i];
    for (int i = tid; i < NP; i += NTH) sNu[i] = A.nu ? A.nu[e * NP + i] : 0.0;
    for (int i = tid; i < NT; i += NTH) {
        int f = i / (M * NFP), rem = i - f * M * NFP, a = rem / NFP, l = rem - a * NFP;
        int64_t F = A.e2f[e * NF + f];
        sUH[i] = A.UH[(F * M + a) * NFP + A.perm[(e * NF + f) * NFP + l]];
    }
    for (int i = tid; i < GEO; i += NTH) geo[i] = A.geo[e * GEO + i];
    __syncthreads();
    const double detJ = geo[0];
    const double* Jinv = geo + 1;
    const double* NW = geo + 1 + D * D;
    // Q_lift = M^{-1}(-C U + E Uhat), so R_q = M (Q - Q_lift) (eq. hdg-grad)
    for (int idx = tid; idx < M * NP; idx += NTH) {
        int a = idx / NP, i = idx - a * NP;
        double ql[D];
        lift_at_node<C>(T, sU, sUH, Jinv, NW, detJ, a, i, ql);
        for (int l = 0; l < D; ++l) sQL[(l * M + a) * NP + i] = sQ[(l * M + a) * NP + i] - ql[l];   // Q - Q_lift
    }
    const PhysT<double>& ph = A.ph;
    for (int g = tid; g < NQ; g += NTH) {
        double u[M], q[M][D], nuv = 0.0;
        for (int a = 0; a < M; ++a) { u[a] = 0.0; for (int l = 0; l < D; ++l) q[a][l] = 0.0; }
        for (int j = 0; j < NP; ++j) {
            double w = T.phi[g * NP + j];
            nuv += w * sNu[j];
            for (int a = 0; a < M; ++a) {
                u[a] += w * sU[a * NP + j];
                for (int l = 0; l < D; ++l) q[a][l] += w * sQ[(l * M + a) * NP + j];
            }
        }
        const double wJ = -A.dt * T.wq[g] * detJ;
        double Fc[M][D], Fv[M][D];
        conv_flux<D, double, double>(u, ph, Fc);
        visc_flux<D, double, double>(u, q, nuv, ph, Fv);
        for (int r = 0; r < D; ++r)
            for (int a = 0; a < M; ++a) {
                double s = 0.0;
                for (int k = 0; k < D; ++k) s += Jinv[r * D + k] * (Fc[a][k] - Fv[a][k]);
                sF[(r * M + a) * NQ + g] = wJ * s;
            }
    }
    for (int fs = tid; fs < NF * NFQ; fs += NTH) {
        const int f = fs / NFQ, s = fs - f * NFQ;
        double u[M], uh[M], q[M][D], nuv = 0.0;
        for (int a = 0; a < M; ++a) { u[a] = 0.0; uh[a] = 0.0; for (int l = 0; l < D; ++l) q[a][l] = 0.0; }
        for (int lam = 0; lam < NFP; ++lam) {
            double w = T.mu[s * NFP + lam];
            int j = T.fnode[f * NFP + lam];
            nuv += w * sNu[j];
            for (int a = 0; a < M; ++a) {
                u[a] += w * sU[a * NP + j];
                uh[a] += w * sUH[(f * M + a) * NFP + lam];
                for (int l = 0; l < D; ++l) q[a][l] += w * sQ[(l * M + a) * NP + j];
            }
        }
        const double* nw = NW + f * D;
        double nrm = 0.0;
        for (int k = 0; k < D; ++k) nrm += nw[k] * nw[k];
        nrm = sqrt(nrm);
        double tau_s = A.tau;
        if (A.tau_mode) {
            double nh[D];
            for (int k = 0; k < D; ++k) nh[k] = nw[k] / nrm;
            tau_s = stab_tau<D, double, double>(uh, nh, 1.0 / pow(double(1 << D) * detJ, 1.0 / D), ph);
        }
        double Fc[M][D], Fv[M][D];
        conv_flux<D, double, double>(uh, ph, Fc);
        visc_flux<D, double, double>(uh, q, nuv, ph, Fv);
        const int tag = A.ftag ? A.ftag[e * NF + f] : 0;
        for (int a = 0; a < M; ++a) {
            double fn = 0.0;
            for (int k = 0; k < D; ++k) fn += (Fc[a][k] - Fv[a][k]) * nw[k];
            const double fh = T.wf[s] * (fn + nrm * tau_s * (u[a] - uh[a]));
            sFH[(f * M + a) * NFQ + s] = fh;
            const double ub_a = tag == 1 ? boundary_state<NF, M, NFP>(A.ub, A.ubf, A.e2f, A.perm, T.mu, e, f, s, a) : 0.0;
            sFB[(f * M + a) * NFQ + s] = boundary_form<M>(tag, a, fh, T.wf[s] * nrm, u, uh, ub_a, A.ew);
        }
    }
    __syncthreads();
    for (int idx = tid; idx < NT; idx += NTH) {
        int f = idx / (M * NFP), rem = idx - f * M * NFP, a = rem / NFP, l = rem - a * NFP;
        double s = 0.0, sb = 0.0;
        for (int q = 0; q < NFQ; ++q) {
            s += T.mu[q * NFP + l] * sFH[(f * M + a) * NFQ + q];
            sb += T.mu[q * NFP + l] * sFB[(f * M + a) * NFQ + q];
        }
        sRh[idx] = s;
        A.rk[e * NT + idx] = (A.ftag && A.ftag[e * NF + f] != 0) ? sb : s;
    }
    __syncthreads();
    double ss = 0.0;
    for (int idx = tid; idx < NU; idx += NTH) {
        int a = idx / NP, i = idx - a * NP;
        double mass = 0.0;
        for (int j = 0; j < NP; ++j) mass += T.mhat[i * NP + j] * (sU[a * NP + j] - A.Ustar[e * NU + a * NP + j]);
        double s = mass * detJ / A.a_ii;
        for (int r = 0; r < D; ++r)
            for (int g = 0; g < NQ; ++g) s += T.dphi[((size_t)r * NQ + g) * NP + i] * sF[(r * M + a) * NQ + g];
        for (int k = 0; k < D; ++k) {
            int nfc = T.node_face[i * D + k];
            if (nfc < 0) continue;
            int f = nfc / NFP, l = nfc - f * NFP;
            s += A.dt * sRh[(f * M + a) * NFP + l];
        }
        if (A.Ru) A.Ru[e * NU + idx] = s;
        ss += s * s;
    }
    for (int idx = tid; idx < NQV; idx += NTH) {
        int la = idx / NP, i = idx - la * NP;
        double s = 0.0;
        for (int j = 0; j < NP; ++j) s += T.mhat[i * NP + j] * sQL[la * NP + j];
        s *= detJ;
        if (A.Rq) A.Rq[e * NQV + idx] = s;
        ss += s * s;
    }
    // fixed-order block reduction
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, off);
    if ((tid & 31) == 0) red[tid >> 5] = ss;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < NTH / 32; ++w) t += red[w];
        A.part[e] = t;
    }
}

// R_uhat[F] = sum over the face's elements (ascending) of their contributions
template <class C>
__global__ void k_trace_residual(const double* rk, const int32_t* f2e, const int32_t* f2lf, const int32_t* iperm,
                                 double* Ruh, double* part, int64_t F) {
    constexpr int M = C::M, NF = C::NF, NFP = C::NFP, NT = C::NT, BS = C::BS;
    const int64_t f = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (f >= F) return;
    double ss = 0.0;
    for (int idx = lane; idx < BS; idx += 32) {
        int a = idx / NFP, k = idx - a * NFP;
        double s = 0.0;
        for (int side = 0; side < 2; ++side) {
            int32_t e = f2e[2 * f + side];
            if (e < 0) continue;
            int fl = f2lf[2 * f + side];
            int l = iperm[((size_t)e * NF + fl) * NFP + k];
            s += rk[(size_t)e * NT + (fl * M + a) * NFP + l];
        }
        if (Ruh) Ruh[f * BS + idx] = s;
        ss += s * s;
    }
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, off);
    if (lane == 0) part[f] = ss;
}

// ----------------------------------------------------------------------------
// block-Jacobi: the explicit inverses of the diagonal blocks S_FF (LU with
// partial pivoting in FP64, then one triangular solve pair per unit column),
// stored column-major in the system's storage type (FP64, or FP32 for the
// mixed system); the apply is then one dense product per face with a
// coalesced column sweep and no reductions.
// ----------------------------------------------------------------------------
template <class C, class TL>
__global__ void k_bj_setup(const int32_t* rowptr, const int32_t* col, const TL* vals, TL* inv, int32_t* status) {
    constexpr int BS = C::BS, LDA = BS + 1;
    extern __shared__ double a[];          // [BS][BS + 1]
    __shared__ int p_s;
    __shared__ int pv_s[BS];
    const int64_t f = blockIdx.x;
    int bd = -1;
    for (int b = rowptr[f]; b < rowptr[f + 1]; ++b)
        if (col[b] == f) bd = b;
    if (bd < 0) {                          // cannot happen for a valid pattern
        if (threadIdx.x == 0) atomicOr(status, 1);
        return;
    }
    const TL* v = vals + (size_t)bd * BS * BS;      // column-major block
    for (int idx = threadIdx.x; idx < BS * BS; idx += blockDim.x) {
        int c = idx / BS, r = idx - c * BS;
        a[r * LDA + c] = (double)v[idx];
    }
    __syncthreads();
    for (int j = 0; j < BS; ++j) {
        if (threadIdx.x == 0) {
            int pr = j;
            double bv = fabs(a[j * LDA + j]);
            for (int r = j + 1; r < BS; ++r)
                if (fabs(a[r * LDA + j]) > bv) { bv = fabs(a[r * LDA + j]); pr = r; }
            if (bv == 0.0 || !isfinite(bv)) atomicOr(status, bv == 0.0 ? 1 : 2);
            p_s = pr;
            pv_s[j] = pr;
        }
        __syncthreads();
        const int pr = p_s;
        if (pr != j)
            for (int c = threadIdx.x; c < BS; c += blockDim.x) {
                double t = a[j * LDA + c]; a[j * LDA + c] = a[pr * LDA + c]; a[pr * LDA + c] = t;
            }
        __syncthreads();
        double pv = a[j * LDA + j];
        if (pv == 0.0 || !isfinite(pv)) pv = 1.0;
        for (int r = j + 1 + threadIdx.x; r < BS; r += blockDim.x) {
            double l = a[r * LDA + j] / pv;
            a[r * LDA + j] = l;
            for (int c = j + 1; c < BS; ++c) a[r * LDA + c] = fma(-l, a[j * LDA + c], a[r * LDA + c]);
        }
        __syncthreads();
    }
    // column c of the inverse: x = U^{-1} L^{-1} P e_c, one thread per column
    TL* out = inv + (size_t)f * BS * BS;
    for (int c = threadIdx.x; c < BS; c += blockDim.x) {
        double x[BS];
        for (int i = 0; i < BS; ++i) x[i] = (i == c) ? 1.0 : 0.0;
        for (int j = 0; j < BS; ++j) {
            const int pr = pv_s[j];
            if (pr != j) { const double t = x[j]; x[j] = x[pr]; x[pr] = t; }
        }
        for (int j = 0; j < BS; ++j)
            for (int i = j + 1; i < BS; ++i) x[i] = fma(-a[i * LDA + j], x[j], x[i]);
        for (int j = BS - 1; j >= 0; --j) {
            double d = a[j * LDA + j];
            if (d == 0.0 || !isfinite(d)) d = 1.0;
            x[j] /= d;
            for (int i = 0; i < j; ++i) x[i] = fma(-a[i * LDA + j], x[j], x[i]);
        }
        for (int i = 0; i < BS; ++i) out[(size_t)c * BS + i] = (TL)x[i];
    }
}

// y_F = inv(S_FF) x_F: one warp per face, lane i owns rows i, i + 32, ...
template <class C, class TL>
__global__ void k_bj_apply(const TL* inv, const double* x, double* y, int64_t F) {
    constexpr int BS = C::BS, RPL = (BS + 31) / 32;
    const int64_t f = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (f >= F) return;
    __shared__ TL buf[8][BS];
    TL* z = buf[threadIdx.x >> 5];
    for (int i = lane; i < BS; i += 32) z[i] = (TL)x[f * BS + i];
    __syncwarp();
    const TL* A = inv + (size_t)f * BS * BS;
    TL acc[RPL];
#pragma unroll
    for (int r = 0; r < RPL; ++r) acc[r] = (TL)0;
    for (int j = 0; j < BS; ++j) {
        const TL zj = z[j];
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
            const int i = lane + 32 * r;
            if (i < BS) acc[r] = fma(A[(size_t)j * BS + i], zj, acc[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        const int i = lane + 32 * r;
        if (i < BS) y[f * BS + i] = (double)acc[r];
    }
}

// ----------------------------------------------------------------------------
// vector kernels (FP64, deterministic reductions)
// ----------------------------------------------------------------------------
constexpr int kRedBlocks = 304;  // 2 per SM
constexpr int kMaxBasis = 512;   // Krylov basis vectors (restart + 1 <= 501)

__global__ void k_dot_part(const double* x, const double* y, int64_t n, double* part);
__global__ void k_dot_final(const double* part, int nparts, double* out, int take_sqrt);
__global__ void k_axpy_dev(const double* coef, double sign, const double* x, double* y, int64_t n);
__global__ void k_mdot_part(const double* V, int64_t ldv, int k, const double* w, int64_t n, double* part);
__global__ void k_mdot_final(const double* part, int nparts, int k, double* out);
__global__ void k_msub(const double* V, int64_t ldv, const double* coef, int k, double* w, int64_t n);
__global__ void k_vadd(double* a, const double* b, int k);
__global__ void k_scale_dev(const double* x, const double* div, double* y, int64_t n);
__global__ void k_axpby(double a, const double* x, double b, double* y, int64_t n);
__global__ void k_combine(const double* V, int64_t ldv, const double* coef, int k, double* x, int64_t n);
__global__ void k_sum_parts(const double* p1, int64_t n1, const double* p2, int64_t n2, double* out);
__global__ void k_scale_safe(const double* x, const double* div, double* y, int64_t n);
__global__ void k_givens_step(const double* hcol, int j, int m, double* R, double* cs, double* sn, double* gv);
__global__ void k_backsolve(const double* R, const double* gv, int k, int m, double* y);
__global__ void k_set_first(const double* beta, double* gv, int m);
__global__ void k_hist_push(const double* norms, double* hist, int* counter, int cap);
__global__ void k_lincomb3(double a, const double* x, double b, const double* y, double c, double* z, int64_t n);
constexpr int kRbMax = 20;            // largest reduced-basis window
constexpr int kRbBlocks = 304;        // row-tile blocks of the Gram reduction
__global__ void k_rb_gram_part(const double* Z, int nb, const double* g, int64_t n, double* part);
__global__ void k_rb_solve(const double* part, int nparts, int nb, double* c);
__global__ void k_rb_store(const double* w, const double* z, double* W, double* Z, const int* head, int64_t n);
__global__ void k_rb_advance(int* head, int nb);

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
template <int D, int P>
int run_residual(hdg_ctx* h, const LinArgs& la, double* Rq, double* Ru, double* Ruh) {
    using C = Cfg<D, P>;
    constexpr int NTH = 128;
    const size_t smem = sizeof(double) * res_smem_doubles<C>();
    HDG_CK(cudaFuncSetAttribute(k_residual<C, NTH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ResArgs ra;
    ra.U = la.U; ra.Q = la.Q; ra.UH = la.UH; ra.Ustar = la.Ustar; ra.nu = la.nu; ra.dt = la.dt; ra.a_ii = la.a_ii;
    ra.ph = phys_t<double>(h->phys); ra.tau = h->phys.tau; ra.tau_mode = h->phys.tau_mode; ra.tab = h->tab; ra.geo = h->d_geo; ra.e2f = h->d_e2f; ra.perm = h->d_perm;
    ra.Rq = Rq; ra.Ru = Ru; ra.rk = h->d_rk; ra.part = h->d_part; ra.ftag = h->d_ftag; ra.ub = h->d_ub;
    ra.ubf = h->d_ubf; ra.ew = h->e_wall;
    k_residual<C, NTH><<<(unsigned)h->E, NTH, smem, h->stream>>>(ra);
    k_trace_residual<C><<<(unsigned)((h->F + 7) / 8), 256, 0, h->stream>>>(h->d_rk, h->d_f2e, h->d_f2lf, h->d_iperm,
                                                                        Ruh, h->d_part + h->E, h->F);
    HDG_CK(cudaGetLastError());
    return HDG_OK;
}

template <int D, int P>
int run_lift(hdg_ctx* h, const double* U, const double* UH, double* Q) {
    using C = Cfg<D, P>;
    k_lift<C, 128><<<(unsigned)h->E, 128, 0, h->stream>>>(U, UH, Q, h->tab, h->d_geo, h->d_e2f, h->d_perm);
    HDG_CK(cudaGetLastError());
    return HDG_OK;
}

template <int D, int P>
int run_bj_setup(hdg_ctx* h) {
    using C = Cfg<D, P>;
    const size_t smem = sizeof(double) * C::BS * (C::BS + 1);
    if (h->sys_prec == HDG_PREC_MIXED) {
        HDG_CK(cudaFuncSetAttribute(k_bj_setup<C, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_bj_setup<C, float><<<(unsigned)h->F, 128, smem, h->stream>>>(h->d_rowptr, h->d_col, h->d_vals32,
                                                                       (float*)h->d_bjlu, h->d_status);
    } else {
        HDG_CK(cudaFuncSetAttribute(k_bj_setup<C, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_bj_setup<C, double><<<(unsigned)h->F, 128, smem, h->stream>>>(h->d_rowptr, h->d_col, h->d_vals,
                                                                        h->d_bjlu, h->d_status);
    }
    h->bj_prec = h->sys_prec;
    HDG_CK(cudaGetLastError());
    return HDG_OK;
}

template <int D, int P>
int run_bj_apply(hdg_ctx* h, const double* x, double* y) {
    using C = Cfg<D, P>;
    if (h->bj_prec == HDG_PREC_MIXED)
        k_bj_apply<C, float><<<(unsigned)((h->F + 7) / 8), 256, 0, h->stream>>>((const float*)h->d_bjlu, x, y, h->F);
    else
        k_bj_apply<C, double><<<(unsigned)((h->F + 7) / 8), 256, 0, h->stream>>>(h->d_bjlu, x, y, h->F);
    HDG_CK(cudaGetLastError());
    return HDG_OK;
}

#define HDG_INSTANTIATE_SOLVE(D, P)                                                       \
    template int run_residual<D, P>(hdg_ctx*, const LinArgs&, double*, double*, double*); \
    template int run_lift<D, P>(hdg_ctx*, const double*, const double*, double*);         \
    template int run_asm_setup<D, P>(hdg_ctx*);                                           \
    template int run_av_field<D, P>(hdg_ctx*, const double*, const double*, double, double, double, double*); \
    template int run_diagnostics<D, P>(hdg_ctx*, const double*, const double*);           \
    template int run_asm_apply<D, P>(hdg_ctx*, const double*, double*);                   \
    template int run_bj_setup<D, P>(hdg_ctx*);                                            \
    template int run_bj_apply<D, P>(hdg_ctx*, const double*, double*);

}  // namespace hdg
