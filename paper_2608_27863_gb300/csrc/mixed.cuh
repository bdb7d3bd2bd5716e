// Mixed-precision condensation.  The interior block At and both right-hand
// sides stay in FP64 and At is factored with partial pivoting in FP64; the
// blocks Bt, Ct, Dt and the condensed trace blocks are FP32.
//
// k_elim_mixed runs the bordered elimination of k_elim on the FP64 part and
// the two FP32 off-diagonal regions, but does not touch Dt: after the last
// panel the interior rows hold [U | Z = L^{-1} P Bt | z = L^{-1} P Rt] and the
// trace rows' multipliers W = Ct U^{-1}, so that the Schur complement is one
// product S^K = Dt - W Z (K = n_u) and -g^K = Rh - W z, left to k_schur_*.
#pragma once

#include "kernels.cuh"

namespace hdg {

// one (up to) 64 x 64 tile of A22 -= L21 U12 in type T; rows/cols >= r_end/c_end skipped
template <int NII, int NJJ, int NB, int TCW, class T, class RowP>
__device__ __forceinline__ void trail_tile_t(RowP rowp, const T* pan, const T* ust, int rb, int ct, int lrow0,
                                             int kb, int tx, int ty, int r_end, int c_end) {
    T acc[NII][NJJ];
    T* rp[NII];
#pragma unroll
    for (int ii = 0; ii < NII; ++ii) {
        int r = rb + ty + 16 * ii;
        rp[ii] = (r < r_end) ? rowp(r) : nullptr;
#pragma unroll
        for (int jj = 0; jj < NJJ; ++jj) {
            int c = ct + tx + 16 * jj;
            acc[ii][jj] = (rp[ii] && c < c_end) ? rp[ii][c] : T(0);
        }
    }
    for (int j = 0; j < kb; ++j) {
        T lv[NII], uv[NJJ];
#pragma unroll
        for (int ii = 0; ii < NII; ++ii) {
            int r = rb + ty + 16 * ii;
            lv[ii] = (r < r_end) ? pan[(size_t)(r - lrow0) * NB + j] : T(0);
        }
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
            if (c < c_end) rp[ii][c] = acc[ii][jj];
        }
    }
}

// trailing update of one storage region: rows [r_begin, r_end) (absolute bordered
// rows, rowp(r) gives the region row), columns [0, c_end) of the region with U12
// row j at urow(j)
template <class T, int NB, int NTH, class RowP, class URow>
__device__ void trailing_region(RowP rowp, URow urow, int r_begin, int r_end, int c_begin, int c_end,
                                const T* pan, int lrow0, int kb, T* ust) {
    constexpr int TCW = 64;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll 1
    for (int ct = c_begin; ct < c_end; ct += TCW) {
        for (int idx = tid; idx < kb * TCW; idx += NTH) {
            int j = idx / TCW, cc = idx - j * TCW;
            ust[j * TCW + cc] = (ct + cc < c_end) ? (T)urow(j)[ct + cc] : T(0);
        }
        __syncthreads();
        int njj = 0;
        while (njj < 4 && ct + 16 * njj < c_end) ++njj;
#pragma unroll 1
        for (int rb = r_begin; rb < r_end; rb += 64) {
            int nii = 0;
            while (nii < 4 && rb + 16 * nii < r_end) ++nii;
            switch (nii * 4 + njj - 5) {
#define HDG_TT(I, J) case (I) * 4 + (J) - 5: trail_tile_t<I, J, NB, TCW, T>(rowp, pan, ust, rb, ct, lrow0, kb, tx, ty, r_end, c_end); break;
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

template <class C, int NB>
constexpr int elim_mixed_smem_bytes() {
    return C::NU * NB * 8 + NB * 64 * 8 +                     // top panel (FP64), U12 staging (FP64)
           (C::NT * NB + C::NU * NB + NB * 64 + NB) * 4;      // bottom panel, top panel copy, staging, pivot row (FP32)
}

template <class C, int NB, int NTH, int MINB = 2>
__global__ void __launch_bounds__(NTH, MINB) k_elim_mixed(Regions<float> R, int64_t e0, int32_t* status) {
    constexpr int NU = C::NU, NT = C::NT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t el = blockIdx.x, e = e0 + el;
    double* A11 = R.a11 + e * R.a11_es;
    float* A12 = R.a12 + e * R.a12_es;
    float* A21 = R.a21 + el * R.a21_es;
    double* rt = R.rt + e * R.rt_es;
    const int64_t s11 = R.a11_rs, s12 = R.a12_rs, s21 = R.a21_rs, srt = R.rt_rs;
    extern __shared__ double sm[];
    double* pan = sm;                                        // [NU][NB]  rows of At (FP64), relative to k0
    double* ust64 = pan + NU * NB;                           // [NB][64]
    float* panb = reinterpret_cast<float*>(ust64 + NB * 64); // [NT][NB]  rows of Ct (FP32)
    float* pant = panb + NT * NB;                            // [NU][NB]  FP32 copy of pan
    float* ust32 = pant + NU * NB;                           // [NB][64]
    float* prow = ust32 + NB * 64;                           // [NB]      pivot row (FP32)
    __shared__ int piv[NB];
    __shared__ int sflag;
    if (tid == 0) sflag = 0;

    for (int k0 = 0; k0 < NU; k0 += NB) {
        const int kb = min(NB, NU - k0), ntop = NU - k0;
#pragma unroll 1
        for (int idx = tid; idx < ntop * kb; idx += NTH) {
            int rr = idx / kb, c = idx - rr * kb;
            pan[rr * NB + c] = A11[(k0 + rr) * s11 + k0 + c];
        }
#pragma unroll 1
        for (int idx = tid; idx < NT * kb; idx += NTH) {
            int rr = idx / kb, c = idx - rr * kb;
            panb[rr * NB + c] = A21[rr * s21 + k0 + c];
        }
        __syncthreads();
        for (int j = 0; j < kb; ++j) {
            // warp 0 alone: pivot search (largest magnitude, lowest row on ties), row
            // interchange inside the panel and the FP32 pivot row; one barrier per step
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
                __syncwarp();
                if (lane < kb) prow[lane] = (float)pan[j * NB + lane];
                if (lane == 0) piv[j] = pr;
            }
            __syncthreads();
            double pv = pan[j * NB + j];
            if (pv == 0.0 || !isfinite(pv)) {
                if (tid == 0) sflag |= (pv == 0.0) ? 1 : 2;
                pv = 1.0;
            }
            const double inv = 1.0 / pv;
            const float invf = (float)inv;
#pragma unroll 1
            for (int rr = j + 1 + tid; rr < ntop; rr += NTH) {       // rows of At: FP64
                double l = pan[rr * NB + j] * inv;
                pan[rr * NB + j] = l;
                for (int c = j + 1; c < kb; ++c) pan[rr * NB + c] = fma(-l, pan[j * NB + c], pan[rr * NB + c]);
            }
#pragma unroll 1
            for (int rr = tid; rr < NT; rr += NTH) {                 // rows of Ct: FP32 multipliers
                float l = panb[rr * NB + j] * invf;
                panb[rr * NB + j] = l;
                for (int c = j + 1; c < kb; ++c) panb[rr * NB + c] = fmaf(-l, prow[c], panb[rr * NB + c]);
            }
            __syncthreads();
        }
#pragma unroll 1
        for (int idx = tid; idx < ntop * kb; idx += NTH) {
            int rr = idx / kb, c = idx - rr * kb;
            A11[(k0 + rr) * s11 + k0 + c] = pan[rr * NB + c];
            pant[rr * NB + c] = (float)pan[rr * NB + c];
        }
#pragma unroll 1
        for (int idx = tid; idx < NT * kb; idx += NTH) {
            int rr = idx / kb, c = idx - rr * kb;
            A21[rr * s21 + k0 + c] = panb[rr * NB + c];
        }
        __syncthreads();
        // interior rows of the trailing columns: swaps, then U12 = L11^{-1} A12
        const int c0 = k0 + kb;
        const int nd = NU - c0 + 1;                               // FP64 columns: At [c0, NU) and Rt
#pragma unroll 1
        for (int cc = tid; cc < nd + NT; cc += NTH) {
            if (cc < nd) {
                double* col = cc < nd - 1 ? A11 + c0 + cc : rt;
                const int64_t st = cc < nd - 1 ? s11 : srt;
                for (int j = 0; j < kb; ++j) {
                    int pr = piv[j];
                    if (pr != j) { double t = col[(k0 + j) * st]; col[(k0 + j) * st] = col[(k0 + pr) * st]; col[(k0 + pr) * st] = t; }
                }
                double xv[NB];
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    if (j < kb) {
                        double s = col[(k0 + j) * st];
#pragma unroll
                        for (int i = 0; i < NB; ++i)
                            if (i < j) s = fma(-pan[j * NB + i], xv[i], s);
                        xv[j] = s;
                        col[(k0 + j) * st] = s;
                    }
                }
            } else {
                float* col = A12 + (cc - nd);
                for (int j = 0; j < kb; ++j) {
                    int pr = piv[j];
                    if (pr != j) { float t = col[(k0 + j) * s12]; col[(k0 + j) * s12] = col[(k0 + pr) * s12]; col[(k0 + pr) * s12] = t; }
                }
                float xv[NB];
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    if (j < kb) {
                        float s = col[(k0 + j) * s12];
#pragma unroll
                        for (int i = 0; i < NB; ++i)
                            if (i < j) s = fmaf(-pant[j * NB + i], xv[i], s);
                        xv[j] = s;
                        col[(k0 + j) * s12] = s;
                    }
                }
            }
        }
        __syncthreads();
        // At (FP64): rows [c0, NU) x cols [c0, NU)
        trailing_region<double, NB, NTH>([&](int r) { return A11 + r * s11; },
                                         [&](int j) { return (const double*)(A11 + (k0 + j) * s11); },
                                         c0, NU, c0, NU, pan, k0, kb, ust64);
        // Ct multipliers (FP32): rows of Ct x cols [c0, NU)
        trailing_region<float, NB, NTH>([&](int r) { return A21 + r * s21; },
                                        [&](int j) { return (const double*)(A11 + (k0 + j) * s11); },
                                        0, NT, c0, NU, panb, 0, kb, ust32);
        // Bt (FP32): rows [c0, NU) x all t columns
        trailing_region<float, NB, NTH>([&](int r) { return A12 + r * s12; },
                                        [&](int j) { return (const float*)(A12 + (k0 + j) * s12); },
                                        c0, NU, 0, NT, pant, k0, kb, ust32);
        // Rt (FP64): rows [c0, NU)
#pragma unroll 1
        for (int r = c0 + tid; r < NU; r += NTH) {
            double s = rt[r * srt];
            for (int j = 0; j < kb; ++j) s = fma(-pan[(r - k0) * NB + j], rt[(k0 + j) * srt], s);
            rt[r * srt] = s;
        }
        __syncthreads();
    }
    if (tid == 0 && sflag) atomicOr(status, sflag);
}

// S^K = Dt - W Z (in place over Dt) and Rh <- Rh - W z, FP32 SIMT with FP32
// accumulation (W [t][n_u] = Ct region, Z [n_u][t] = Bt region after k_elim_mixed)
// ----------------------------------------------------------------------------
// A3 + A4 of the mixed form, split by precision.  k_lu_mixed factors the
// interior block in FP64 alone, P At = L U with partial pivoting (blocked
// panels, pivot step in one warp, LAPACK-style full-row interchanges), and
// forms z = L^{-1} P Rt; it stores the interchanges.  The FP32 border then
// needs two triangular solves with many right-hand sides, each independent
// per column (or row) and run by its own kernels:
//   k_trsm_z:  Z = L^{-1} P Bt   (columns of Bt)
//   k_trsm_w:  W = Ct U^{-1}     (rows of Ct)
// 32-row blocks of the factor are staged in shared memory as FP32; the
// off-diagonal part of each block step is a small product (threads over
// rows x columns), the diagonal 32 x 32 triangle is solved per column.
// ----------------------------------------------------------------------------
template <class C, int NB>
constexpr int lu_mixed_smem_bytes() { return (C::NU * NB + NB * 64) * 8; }

template <class C, int NB, int NTH>
__global__ void __launch_bounds__(NTH, 2) k_lu_mixed(Regions<float> R, int32_t* __restrict__ piv_out,
                                                     int64_t e0, int32_t* status) {
    constexpr int NU = C::NU;
    static_assert(NTH == 256, "trailing-update layout assumes 256 threads");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t e = e0 + blockIdx.x;
    double* A = R.a11 + e * R.a11_es;
    double* rt = R.rt + e * R.rt_es;
    const int64_t rs = R.a11_rs, srt = R.rt_rs;
    auto rowp = [&](int r) -> double* { return A + (size_t)r * rs; };
    extern __shared__ double sm[];
    double* pan = sm;                    // [NU][NB], row index relative to k0
    double* ust = pan + NU * NB;         // [NB][64]
    __shared__ int piv[NB];
    __shared__ int sflag;
    if (tid == 0) sflag = 0;
    __syncthreads();
#pragma unroll 1
    for (int k0 = 0; k0 < NU; k0 += NB) {
        const int kb = min(NB, NU - k0), nrows = NU - k0;
#pragma unroll 1
        for (int idx = tid; idx < nrows * kb; idx += NTH) {
            const int rr = idx / kb, c = idx - rr * kb;
            pan[rr * NB + c] = rowp(k0 + rr)[k0 + c];
        }
        __syncthreads();
#pragma unroll 1
        for (int j = 0; j < kb; ++j) {
            if (warp == 0) {
                double bv = -1.0;
                int bi = INT_MAX;
#pragma unroll 1
                for (int rr = j + lane; rr < nrows; rr += 32) {
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
                const double l = pan[rr * NB + j] * inv;
                pan[rr * NB + j] = l;
                for (int c = j + 1; c < kb; ++c) pan[rr * NB + c] = fma(-l, pan[j * NB + c], pan[rr * NB + c]);
            }
            __syncthreads();
        }
#pragma unroll 1
        for (int idx = tid; idx < nrows * kb; idx += NTH) {
            const int rr = idx / kb, c = idx - rr * kb;
            rowp(k0 + rr)[k0 + c] = pan[rr * NB + c];
        }
        // interchanges outside the panel (factor columns to the left, trailing columns
        // and the right-hand side), then U12 = L11^{-1} A12 and the same for Rt
        const int c0 = k0 + kb;
#pragma unroll 1
        for (int c = tid; c <= NU; c += NTH) {
            if (c >= k0 && c < c0) continue;
            double* col = c < NU ? A + c : rt;
            const int64_t st = c < NU ? rs : srt;
            for (int j = 0; j < kb; ++j) {
                const int pr = piv[j];
                if (pr != j) {
                    const double t = col[(k0 + j) * st];
                    col[(k0 + j) * st] = col[(k0 + pr) * st];
                    col[(k0 + pr) * st] = t;
                }
            }
            if (c >= c0) {
                double xv[NB];
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    if (j < kb) {
                        double s = col[(k0 + j) * st];
#pragma unroll
                        for (int i = 0; i < NB; ++i)
                            if (i < j) s = fma(-pan[j * NB + i], xv[i], s);
                        xv[j] = s;
                        col[(k0 + j) * st] = s;
                    }
                }
            }
        }
        if (tid < kb) piv_out[e * NU + k0 + tid] = k0 + piv[tid];
        __syncthreads();
        trailing_region<double, NB, NTH>(rowp, [&](int j) { return rowp(k0 + j); }, c0, NU, c0, NU, pan, k0, kb, ust);
        // right-hand side: rt[r] -= L21[r] . z1 for the rows below the panel
#pragma unroll 1
        for (int r = c0 + tid; r < NU; r += NTH) {
            double s = rt[r * srt];
            for (int j = 0; j < kb; ++j) s = fma(-pan[(r - k0) * NB + j], rt[(k0 + j) * srt], s);
            rt[r * srt] = s;
        }
        __syncthreads();
    }
    if (tid == 0 && sflag) atomicOr(status, sflag);
}

// X[i0 + r][c] -= sum_{j < i0} F[r][j] X[j][c] for r < nb, c < CW (F a staged factor
// block row, row stride NU): each thread owns a 4-row x 2-column tile, so one pair
// of shared loads feeds eight multiply-adds
template <int NU, int CW, int NTH>
__device__ __forceinline__ void trsm_offdiag_tile(const float* F, float* X, int i0, int nb) {
    static_assert(32 * CW == 8 * NTH, "tile layout assumes 32 x CW outputs over NTH threads");
    const int tid = threadIdx.x, cp = tid % (CW / 2), rq = tid / (CW / 2);
    const int c = 2 * cp, r = 4 * rq;
    float acc[4][2] = {};
    if (i0 > 0) {
        for (int j = 0; j < i0; ++j) {
            const float x0 = X[j * CW + c], x1 = X[j * CW + c + 1];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float f = F[(r + u) * NU + j];
                acc[u][0] = fmaf(f, x0, acc[u][0]);
                acc[u][1] = fmaf(f, x1, acc[u][1]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (r + u < nb) {
                X[(i0 + r + u) * CW + c] -= acc[u][0];
                X[(i0 + r + u) * CW + c + 1] -= acc[u][1];
            }
    }
}

template <class C>
struct TrsmShape {
    static constexpr int CW = 64;                           // right-hand sides per CTA
    static constexpr int NTH = 256;
    static constexpr int smem_floats = C::NU * CW + 32 * C::NU;   // the block of right-hand sides, one factor block row
};

// Z = L^{-1} P Bt for columns [c0, c0 + CW) of Bt (FP32, in place); L unit lower (FP64 storage)
template <class C>
__global__ void __launch_bounds__(TrsmShape<C>::NTH) k_trsm_z(Regions<float> R, const int32_t* __restrict__ piv,
                                                              int64_t e0) {
    constexpr int NU = C::NU, NT = C::NT, CW = TrsmShape<C>::CW, NTH = TrsmShape<C>::NTH;
    constexpr int NCT = (NT + CW - 1) / CW;
    const int tid = threadIdx.x;
    const int64_t e = e0 + blockIdx.x / NCT;
    const int c0 = (int)(blockIdx.x % NCT) * CW;
    const int cw = min(CW, NT - c0);
    const double* A = R.a11 + e * R.a11_es;
    float* Bt = R.a12 + e * R.a12_es;
    const int64_t rs = R.a11_rs, bs = R.a12_rs;
    extern __shared__ float smf[];
    float* X = smf;                       // [NU][CW]
    float* Lb = X + NU * CW;              // [32][NU] one block row of L
    __shared__ int perm[NU];
    if (tid == 0) {                       // the interchange sequence as a gather map
        for (int i = 0; i < NU; ++i) perm[i] = i;
        for (int i = 0; i < NU; ++i) {
            const int q = piv[e * NU + i];
            if (q != i) { const int t = perm[i]; perm[i] = perm[q]; perm[q] = t; }
        }
    }
    __syncthreads();
    for (int idx = tid; idx < NU * CW; idx += NTH) {
        const int i = idx / CW, c = idx - i * CW;
        X[idx] = c < cw ? Bt[(size_t)perm[i] * bs + c0 + c] : 0.f;
    }
#pragma unroll 1
    for (int i0 = 0; i0 < NU; i0 += 32) {
        const int nb = min(32, NU - i0);
        __syncthreads();
        for (int idx = tid; idx < nb * (i0 + nb); idx += NTH) {
            const int r = idx / (i0 + nb), j = idx - r * (i0 + nb);
            Lb[r * NU + j] = (float)A[(size_t)(i0 + r) * rs + j];
        }
        __syncthreads();
        // X[i0 + r][c] -= sum_{j < i0} L[i0 + r][j] X[j][c]: each thread a 4 x 2 tile
        trsm_offdiag_tile<NU, CW, NTH>(Lb, X, i0, nb);
        __syncthreads();
        // the unit-lower diagonal block, one column per thread, the column in registers
        for (int c = tid; c < CW; c += NTH) {
            float x[32];
#pragma unroll
            for (int r = 0; r < 32; ++r) x[r] = r < nb ? X[(i0 + r) * CW + c] : 0.f;
#pragma unroll
            for (int r = 1; r < 32; ++r) {
                float s = x[r];
#pragma unroll
                for (int j = 0; j < 32; ++j)      // rows past nb read nothing: the staged block ends there
                    if (j < r && r < nb) s = fmaf(-Lb[r * NU + i0 + j], x[j], s);
                x[r] = r < nb ? s : 0.f;
            }
#pragma unroll
            for (int r = 0; r < 32; ++r)
                if (r < nb) X[(i0 + r) * CW + c] = x[r];
        }
    }
    __syncthreads();
    for (int idx = tid; idx < NU * CW; idx += NTH) {
        const int i = idx / CW, c = idx - i * CW;
        if (c < cw) Bt[(size_t)i * bs + c0 + c] = X[idx];
    }
}

// W = Ct U^{-1} for rows [r0, r0 + CW) of Ct (FP32, in place, chunk-local); U upper (FP64 storage)
template <class C>
__global__ void __launch_bounds__(TrsmShape<C>::NTH) k_trsm_w(Regions<float> R, int64_t e0) {
    constexpr int NU = C::NU, NT = C::NT, CW = TrsmShape<C>::CW, NTH = TrsmShape<C>::NTH;
    constexpr int NCT = (NT + CW - 1) / CW;
    const int tid = threadIdx.x;
    const int64_t el = blockIdx.x / NCT, e = e0 + el;
    const int r0 = (int)(blockIdx.x % NCT) * CW;
    const int rw = min(CW, NT - r0);
    const double* A = R.a11 + e * R.a11_es;
    float* Ct = R.a21 + el * R.a21_es;
    const int64_t rs = R.a11_rs, cs = R.a21_rs;
    extern __shared__ float smf[];
    float* X = smf;                       // [NU][CW]: X[j][r] = Ct[r0 + r][j]
    float* Ub = X + NU * CW;              // [32][NU]: Ub[q][j] = U[j][i0 + q], j < i0 + nb
    for (int idx = tid; idx < NU * CW; idx += NTH) {
        const int r = idx / NU, j = idx - r * NU;
        X[j * CW + r] = r < rw ? Ct[(size_t)(r0 + r) * cs + j] : 0.f;
    }
#pragma unroll 1
    for (int i0 = 0; i0 < NU; i0 += 32) {
        const int nb = min(32, NU - i0);
        __syncthreads();
        for (int idx = tid; idx < (i0 + nb) * nb; idx += NTH) {
            const int j = idx / nb, q = idx - j * nb;
            Ub[q * NU + j] = (float)A[(size_t)j * rs + i0 + q];
        }
        __syncthreads();
        // X[i0 + q][r] -= sum_{j < i0} U[j][i0 + q] X[j][r]: each thread a 4 x 2 tile
        trsm_offdiag_tile<NU, CW, NTH>(Ub, X, i0, nb);
        __syncthreads();
        for (int r = tid; r < CW; r += NTH) {
            float x[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) x[q] = q < nb ? X[(i0 + q) * CW + r] : 0.f;
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                float s = x[q];
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j < q && q < nb) s = fmaf(-Ub[q * NU + i0 + j], x[j], s);
                const float d = q < nb ? Ub[q * NU + i0 + q] : 1.f;
                x[q] = q < nb ? s / (d != 0.f ? d : 1.f) : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 32; ++q)
                if (q < nb) X[(i0 + q) * CW + r] = x[q];
        }
    }
    __syncthreads();
    for (int idx = tid; idx < NU * CW; idx += NTH) {
        const int r = idx / NU, j = idx - r * NU;
        if (r < rw) Ct[(size_t)(r0 + r) * cs + j] = X[j * CW + r];
    }
}

template <class C, int NTH>
__global__ void __launch_bounds__(NTH) k_schur_simt(Regions<float> R, int64_t e0) {
    constexpr int NU = C::NU, NT = C::NT, KC = 32, TW = 64;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t el = blockIdx.x, e = e0 + el;
    const float* W = R.a21 + el * R.a21_es;
    const float* Z = R.a12 + e * R.a12_es;
    float* Dm = R.a22 + el * R.a22_es;
    const double* z = R.rt + e * R.rt_es;
    double* rb = R.rb + el * R.rb_es;
    const int64_t sw = R.a21_rs, sz = R.a12_rs, sd = R.a22_rs;
    __shared__ float Ws[TW][KC + 1];
    __shared__ float Zs[KC][TW];
    // right-hand side: rb -= W z (FP64 accumulation)
    for (int r = tid; r < NT; r += NTH) {
        double s = rb[r * R.rb_rs];
        for (int k = 0; k < NU; ++k) s -= (double)W[r * sw + k] * z[k * R.rt_rs];
        rb[r * R.rb_rs] = s;
    }
    for (int rt0 = 0; rt0 < NT; rt0 += TW)
        for (int ct0 = 0; ct0 < NT; ct0 += TW) {
            float acc[4][4];
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[ii][jj] = 0.f;
            for (int k0 = 0; k0 < NU; k0 += KC) {
                for (int idx = tid; idx < TW * KC; idx += NTH) {
                    int r = idx / KC, k = idx - r * KC;
                    Ws[r][k] = (rt0 + r < NT && k0 + k < NU) ? W[(rt0 + r) * sw + k0 + k] : 0.f;
                    int k2 = idx / TW, c = idx - k2 * TW;
                    Zs[k2][c] = (k0 + k2 < NU && ct0 + c < NT) ? Z[(k0 + k2) * sz + ct0 + c] : 0.f;
                }
                __syncthreads();
#pragma unroll 8
                for (int k = 0; k < KC; ++k) {
                    float a[4], b[4];
#pragma unroll
                    for (int ii = 0; ii < 4; ++ii) a[ii] = Ws[ty + 16 * ii][k];
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) b[jj] = Zs[k][tx + 16 * jj];
#pragma unroll
                    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) acc[ii][jj] = fmaf(a[ii], b[jj], acc[ii][jj]);
                }
                __syncthreads();
            }
#pragma unroll
            for (int ii = 0; ii < 4; ++ii) {
                int r = rt0 + ty + 16 * ii;
                if (r >= NT) continue;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    int c = ct0 + tx + 16 * jj;
                    if (c < NT) Dm[r * sd + c] -= acc[ii][jj];
                }
            }
        }
}

// assembly from region views (S^K in Dt, -g^K in Rh) into BSR blocks of type TL
template <class C, class TL>
__global__ void k_assemble_r(Regions<TL> R, int64_t e0, const int32_t* blk, const int32_t* rank,
                             const int32_t* iperm, TL* vals, int pass) {
    constexpr int M = C::M, NF = C::NF, NFP = C::NFP, BS = C::BS;
    const int64_t bid = blockIdx.x;
    const int gl = (int)(bid % NF), fl = (int)((bid / NF) % NF);
    const int64_t el = bid / (NF * NF), e = e0 + el;
    const size_t item = ((size_t)e * NF + fl) * NF + gl;
    if (rank[item] != pass) return;
    TL* out = vals + (size_t)blk[item] * BS * BS;
    const TL* S = R.a22 + el * R.a22_es;
    const int32_t* ipf = iperm + ((size_t)e * NF + fl) * NFP;
    const int32_t* ipg = iperm + ((size_t)e * NF + gl) * NFP;
    for (int idx = threadIdx.x; idx < BS * BS; idx += blockDim.x) {
        int c = idx / BS, r = idx - c * BS;
        int a = r / NFP, k = r - a * NFP, b2 = c / NFP, k2 = c - b2 * NFP;
        int row = (fl * M + a) * NFP + ipf[k];
        int col = (gl * M + b2) * NFP + ipg[k2];
        out[idx] += S[(size_t)row * R.a22_rs + col];
    }
}

template <class C, class TL>
__global__ void k_assemble_g_r(Regions<TL> R, int64_t e0, const int32_t* e2f, const int32_t* frank,
                               const int32_t* iperm, double* g, int pass) {
    constexpr int M = C::M, NF = C::NF, NFP = C::NFP, BS = C::BS;
    const int64_t bid = blockIdx.x;
    const int fl = (int)(bid % NF);
    const int64_t el = bid / NF, e = e0 + el;
    if (frank[e * NF + fl] != pass) return;
    const int64_t F = e2f[e * NF + fl];
    const double* rb = R.rb + el * R.rb_es;
    const int32_t* ipf = iperm + ((size_t)e * NF + fl) * NFP;
    for (int idx = threadIdx.x; idx < BS; idx += blockDim.x) {
        int a = idx / NFP, k = idx - a * NFP;
        int row = (fl * M + a) * NFP + ipf[k];
        g[F * BS + idx] -= rb[row * R.rb_rs];
    }
}

// y = S x with blocks of type TL, FP64 vectors and accumulation
template <class C, class TL>
__global__ void __launch_bounds__(MvShape<C>::NTH) k_matvec_t(const int32_t* rowptr, const int32_t* col,
                                                              const TL* vals, const double* x, double* y) {
    constexpr int BS = C::BS, RB = MvShape<C>::RB, GROUPS = MvShape<C>::GROUPS;
    __shared__ double part[GROUPS][RB];
    const int64_t F = blockIdx.x;
    const int grp = threadIdx.x / RB, r = threadIdx.x - grp * RB;
    double acc0 = 0.0, acc1 = 0.0;
    if (r < BS) {
        for (int b = rowptr[F] + grp; b < rowptr[F + 1]; b += GROUPS) {
            const double* xs = x + (size_t)col[b] * BS;
            const TL* v = vals + (size_t)b * BS * BS + r;
            int c = 0;
#pragma unroll 4
            for (; c + 1 < BS; c += 2) {
                acc0 = fma((double)v[(size_t)c * BS], xs[c], acc0);
                acc1 = fma((double)v[(size_t)(c + 1) * BS], xs[c + 1], acc1);
            }
            if (c < BS) acc0 = fma((double)v[(size_t)c * BS], xs[c], acc0);
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

// y = S x with FP32 blocks and an FP32 copy of x: products and the sum within
// each block in FP32, the sum over a row's blocks in FP64
__global__ void k_to_f32(const double* x, float* y, int64_t n);   // solve_vec.cu

template <class C>
__global__ void __launch_bounds__(MvShape<C>::NTH) k_matvec_f32(const int32_t* rowptr, const int32_t* col,
                                                                const float* vals, const float* x, double* y) {
    constexpr int BS = C::BS, RB = MvShape<C>::RB, GROUPS = MvShape<C>::GROUPS;
    __shared__ double part[GROUPS][RB];
    const int64_t F = blockIdx.x;
    const int grp = threadIdx.x / RB, r = threadIdx.x - grp * RB;
    double acc = 0.0;
    if (r < BS) {
        for (int b = rowptr[F] + grp; b < rowptr[F + 1]; b += GROUPS) {
            const float* xs = x + (size_t)col[b] * BS;
            const float* v = vals + (size_t)b * BS * BS + r;
            float a0 = 0.f, a1 = 0.f;
            int c = 0;
#pragma unroll 4
            for (; c + 1 < BS; c += 2) {
                a0 = fmaf(v[(size_t)c * BS], xs[c], a0);
                a1 = fmaf(v[(size_t)(c + 1) * BS], xs[c + 1], a1);
            }
            if (c < BS) a0 = fmaf(v[(size_t)c * BS], xs[c], a0);
            acc += (double)(a0 + a1);
        }
    }
    part[grp][r] = acc;
    __syncthreads();
    if (grp == 0 && r < BS) {
        double s = part[0][r];
        for (int g2 = 1; g2 < GROUPS; ++g2) s += part[g2][r];
        y[F * BS + r] = s;
    }
}

// recovery from region views: dU = -U^{-1}(z + Z dUhat), dQ = dq0 - L dU + Lambda dUhat
template <class C, class TL, int NTH>
__global__ void __launch_bounds__(NTH) k_recover_r(Regions<TL> R, RecArgs A) {
    constexpr int D = C::D, M = C::M, NP = C::NP, NF = C::NF, NFP = C::NFP;
    constexpr int NU = C::NU, NQV = C::NQV, NT = C::NT;
    constexpr int GEO = Geo<D>::N;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t e = blockIdx.x;
    __shared__ double duh[NT];
    __shared__ double w[NU];
    __shared__ double x[NU];
    __shared__ double geo[GEO];
    for (int i = tid; i < NT; i += NTH) {
        int f = i / (M * NFP), rem = i - f * M * NFP, a = rem / NFP, l = rem - a * NFP;
        int64_t F = A.e2f[e * NF + f];
        int k = A.perm[(e * NF + f) * NFP + l];
        duh[i] = A.dUH[(F * M + a) * NFP + k];
    }
    for (int i = tid; i < GEO; i += NTH) geo[i] = A.geo[e * GEO + i];
    __syncthreads();
    const double* U11 = R.a11 + e * R.a11_es;
    const TL* Z = R.a12 + e * R.a12_es;
    const double* z = R.rt + e * R.rt_es;
    // w = Z dUhat + z: each lane sums its products in the storage type (Z is FP32), the
    // lanes' partial sums are combined in FP64 (FP64 work would bound the kernel on GB300)
    for (int i = warp; i < NU; i += NTH / 32) {
        const TL* row = Z + (size_t)i * R.a12_rs;
        TL p = (TL)0;
        for (int c = lane; c < NT; c += 32) p = fma(row[c], (TL)duh[c], p);
        double s = (double)p;
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) w[i] = s + z[i * R.rt_rs];
    }
    __syncthreads();
    // x = U^{-1} w (FP64): 32-row diagonal blocks solved by warp 0 from registers, the
    // rows above updated with one dot product per row and thread
#pragma unroll 1
    for (int k1 = NU; k1 > 0; k1 -= 32) {
        const int k0 = max(0, k1 - 32), nb = k1 - k0;
        if (warp == 0) {
            double ur[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) ur[j] = (lane < nb && j < nb) ? U11[(size_t)(k0 + lane) * R.a11_rs + k0 + j] : 0.0;
            double v = lane < nb ? w[k0 + lane] : 0.0;
#pragma unroll
            for (int j = 31; j >= 0; --j) {
                if (j < nb) {
                    if (lane == j) v = v / ur[j];
                    const double xj = __shfl_sync(0xffffffffu, v, j);
                    if (lane < j) v = fma(-ur[j], xj, v);
                }
            }
            if (lane < nb) x[k0 + lane] = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int r = tid; r < k0; r += NTH) {
            const double* row = U11 + (size_t)r * R.a11_rs + k0;
            double s = 0.0;
            for (int j = 0; j < nb; ++j) s = fma(row[j], x[k0 + j], s);
            w[r] -= s;
        }
        __syncthreads();
    }
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
            for (int j = 0; j < NP; ++j) s -= mc[j] * x[b * NP + j];
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

}  // namespace hdg

namespace hdg {

template <class C, bool SPLIT3>
__global__ void k_schur_tc(Regions<float> R, int64_t e0, int32_t* status);
template <class C>
struct SchurTC;
template <class C>
struct BlkTC;
template <class C>
__global__ void k_blocks_tc(BlkArgs<float> A, int32_t* status);

inline Regions<float> mixed_regions(hdg_ctx* h) {
    const int64_t NU = h->NU, NT = h->NT;
    Regions<float> R;
    R.a11 = h->d_m11; R.a11_es = NU * NU; R.a11_rs = NU;
    R.a12 = h->d_m12; R.a12_es = NU * NT; R.a12_rs = NT;
    R.a21 = h->d_m21; R.a21_es = NT * NU; R.a21_rs = NU;
    R.a22 = h->d_m22; R.a22_es = NT * NT; R.a22_rs = NT;
    R.rt = h->d_mrt;  R.rt_es = NU;       R.rt_rs = 1;
    R.rb = h->d_mrb;  R.rb_es = NT;       R.rb_rs = 1;
    return R;
}

template <int D, int P>
int run_linearize_mixed(hdg_ctx* h, const LinArgs& la) {
    using C = Cfg<D, P>;
    using BC = BlkCfg<C>;
    using BS_ = BlkShape<C, BC::TY, BC::TX, BC::KC>;
    constexpr int PT = 128, NB = 16;
    int rc;
    if ((rc = ensure_system_storage(h, HDG_PREC_MIXED))) return rc;
    auto kblk = k_blocks<C, BC::TY, BC::TX, BC::KC, float, float>;
    auto kface = k_blocks<C, BC::TY, BC::TX, BC::KC, float, float, false>;
    const size_t sm_point = sizeof(double) * point_smem_doubles<C>();
    const size_t sm_blk = sizeof(float) * BS_::smem_f32;
    const size_t sm_elim = elim_mixed_smem_bytes<C, NB>();
    HDG_CK(cudaFuncSetAttribute(k_point<C, PT, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_point));
    HDG_CK(cudaFuncSetAttribute(kblk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_blk));
    HDG_CK(cudaFuncSetAttribute(kface, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_blk));
    if (C::D == 3)
        HDG_CK(cudaFuncSetAttribute(k_blocks_tc<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, BlkTC<C>::smem_bytes()));
    const size_t sm_sf32 = sizeof(float) * SfShape<C, float>::smem_words;
    HDG_CK(cudaFuncSetAttribute(k_blocks_sf<C, float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_sf32));
    HDG_CK(cudaFuncSetAttribute(k_elim_mixed<C, NB, 256, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_elim));
    HDG_CK(cudaFuncSetAttribute(k_elim_mixed<C, NB, 256, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_elim));
    const int sm_lu = lu_mixed_smem_bytes<C, NB>();   // the 8-column variant needs less
    const int sm_trsm = (int)sizeof(float) * TrsmShape<C>::smem_floats;
    HDG_CK(cudaFuncSetAttribute(k_lu_mixed<C, NB, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_lu));
    HDG_CK(cudaFuncSetAttribute(k_lu_mixed<C, 8, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_lu));
    HDG_CK(cudaFuncSetAttribute(k_trsm_z<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_trsm));
    HDG_CK(cudaFuncSetAttribute(k_trsm_w<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_trsm));
    cudaStream_t st = h->stream;
    HDG_CK(cudaMemsetAsync(h->d_vals32, 0, sizeof(float) * h->nnzb * C::BS * C::BS, st));
    HDG_CK(cudaMemsetAsync(h->d_g, 0, sizeof(double) * h->F * C::BS, st));
    const Regions<float> RM = mixed_regions(h);
    PointArgs pa;
    pa.U = la.U; pa.Q = la.Q; pa.UH = la.UH; pa.Ustar = la.Ustar; pa.nu = la.nu;
    pa.dt = la.dt; pa.a_ii = la.a_ii; pa.ph = phys_t<double>(h->phys); pa.phf = phys_t<float>(h->phys);
    pa.tau = h->phys.tau; pa.tab = h->tab; pa.geo = h->d_geo;
    pa.e2f = h->d_e2f; pa.perm = h->d_perm;
    pa.rt = RM.rt; pa.rt_es = RM.rt_es; pa.rt_rs = RM.rt_rs;
    pa.rb = RM.rb; pa.rb_es = RM.rb_es; pa.rb_rs = RM.rb_rs;
    pa.vcoef = h->d_vcoef; pa.fcoef = h->d_fcoef; pa.dq0 = h->d_dq0;
    pa.ftag = h->d_ftag; pa.ub = h->d_ub; pa.ubf = h->d_ubf; pa.ew = h->e_wall;
    pa.tau_mode = h->phys.tau_mode; pa.taup = h->phys.tau_mode ? h->d_taup : nullptr;
    BlkArgs<float> ba;
    ba.vcoef = h->d_vcoef; ba.fcoef = h->d_fcoef; ba.geo = h->d_geo; ba.tab = h->tab; ba.ftag = h->d_ftag;
    ba.ew = h->e_wall;
    ba.taup = h->phys.tau_mode ? h->d_taup : nullptr;
    ba.R = RM; ba.dt = la.dt; ba.a_ii = la.a_ii; ba.tau = h->phys.tau;
    for (int64_t e0 = 0; e0 < h->E; e0 += h->chunk) {
        const int64_t ne = std::min<int64_t>(h->chunk, h->E - e0);
        pa.e0 = e0; ba.e0 = e0;
        prof_begin(h, HDG_K_POINT);
        k_point<C, PT, float><<<(unsigned)ne, PT, sm_point, st>>>(pa);
        prof_end(h);
        prof_begin(h, HDG_K_BLOCKS);
        if (h->blocks_mode == 1 && C::D == 3) {
            // volume contraction on tensor cores (3xTF32), face terms added by the SIMT kernel
            using BT = BlkTC<C>;
            k_blocks_tc<C><<<(unsigned)(ne * BT::NMT), BT::THREADS, BT::smem_bytes(), st>>>(ba, h->d_status);
            kface<<<(unsigned)(ne * C::M * C::M), BC::TY * BC::TX, sm_blk, st>>>(ba);
        } else if (h->blocks_mode == 2) {
            // volume contraction by FP32 sum factorisation, then the face terms
            k_blocks_sf<C, float, float><<<(unsigned)(ne * C::M * C::M), SfShape<C, float>::NTH, sm_sf32, st>>>(ba);
            kface<<<(unsigned)(ne * C::M * C::M), BC::TY * BC::TX, sm_blk, st>>>(ba);
        } else {
            kblk<<<(unsigned)(ne * C::M * C::M), BC::TY * BC::TX, sm_blk, st>>>(ba);
        }
        prof_end(h);
        prof_begin(h, HDG_K_ELIM);
        if (h->elim_mixed_split) {
            // FP64 interior LU alone, then the FP32 border by two triangular solves
            using TS = TrsmShape<C>;
            constexpr int NCT = (C::NT + TS::CW - 1) / TS::CW;
            if (h->elim_nb == 8)   // interior LU panel width (the autotuner's elim_nb)
                k_lu_mixed<C, 8, 256><<<(unsigned)ne, 256, sm_lu, st>>>(RM, h->d_mpiv, e0, h->d_status);
            else
                k_lu_mixed<C, NB, 256><<<(unsigned)ne, 256, sm_lu, st>>>(RM, h->d_mpiv, e0, h->d_status);
            k_trsm_z<C><<<(unsigned)(ne * NCT), TS::NTH, sm_trsm, st>>>(RM, h->d_mpiv, e0);
            k_trsm_w<C><<<(unsigned)(ne * NCT), TS::NTH, sm_trsm, st>>>(RM, e0);
        } else if (h->elim_mixed_minb == 3) {  // fused kernel, built for 3 or 2 resident CTAs per SM
            k_elim_mixed<C, NB, 256, 3><<<(unsigned)ne, 256, sm_elim, st>>>(RM, e0, h->d_status);
        } else {
            k_elim_mixed<C, NB, 256, 2><<<(unsigned)ne, 256, sm_elim, st>>>(RM, e0, h->d_status);
        }
        prof_end(h);
        prof_begin(h, HDG_K_SCHUR);
        if (h->schur_mode == 0) {
            k_schur_simt<C, 256><<<(unsigned)ne, 256, 0, st>>>(RM, e0);
        } else {
            using ST = SchurTC<C>;
            const unsigned grid = (unsigned)(ne * ST::NMT * ST::NNT);
            if (h->schur_mode == 1) {
                const int smb = ST::smem_bytes(false);
                HDG_CK(cudaFuncSetAttribute(k_schur_tc<C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
                k_schur_tc<C, false><<<grid, ST::THREADS, smb, st>>>(RM, e0, h->d_status);
            } else {
                const int smb = ST::smem_bytes(true);
                HDG_CK(cudaFuncSetAttribute(k_schur_tc<C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
                k_schur_tc<C, true><<<grid, ST::THREADS, smb, st>>>(RM, e0, h->d_status);
            }
        }
        prof_end(h);
        if (h->d_skout)
            k_copy_sk<float, float><<<(unsigned)ne, 256, 0, st>>>(RM.a22, RM.a22_es, RM.a22_rs, 0, C::NT, e0,
                                                                  static_cast<float*>(h->d_skout));
        for (int pass = 0; pass < 2; ++pass) {
            prof_begin(h, HDG_K_ASSEMBLE);
            k_assemble_r<C, float><<<(unsigned)(ne * C::NF * C::NF), 256, 0, st>>>(RM, e0, h->d_blk, h->d_rank,
                                                                                 h->d_iperm, h->d_vals32, pass);
            prof_end(h);
            prof_begin(h, HDG_K_ASSEMBLE);
            k_assemble_g_r<C, float><<<(unsigned)(ne * C::NF), 128, 0, st>>>(RM, e0, h->d_e2f, h->d_frank,
                                                                            h->d_iperm, h->d_g, pass);
            prof_end(h);
        }
        HDG_CK(cudaGetLastError());
    }
    h->have_system = true;
    h->sys_prec = HDG_PREC_MIXED;
    h->bj_ready = false;
    h->asm_ready = false;
    return HDG_OK;
}

template <int D, int P>
int run_matvec(hdg_ctx* h, const double* x, double* y) {
    using C = Cfg<D, P>;
    prof_begin(h, HDG_K_MATVEC);
    if (h->sys_prec == HDG_PREC_MIXED) {
        const int64_t n = h->F * C::BS;
        k_to_f32<<<(unsigned)std::min<int64_t>(1216, (n + 255) / 256), 256, 0, h->stream>>>(x, h->d_x32, n);
        k_matvec_f32<C><<<(unsigned)h->F, MvShape<C>::NTH, 0, h->stream>>>(h->d_rowptr, h->d_col, h->d_vals32,
                                                                          h->d_x32, y);
    } else
        k_matvec<C><<<(unsigned)h->F, MvShape<C>::NTH, 0, h->stream>>>(h->d_rowptr, h->d_col, h->d_vals, x, y);
    prof_end(h);
    HDG_CK(cudaGetLastError());
    return HDG_OK;
}

template <int D, int P>
int run_recover_mixed(hdg_ctx* h, const double* dUH, double* dQ, double* dU) {
    using C = Cfg<D, P>;
    RecArgs ra;
    ra.top = nullptr; ra.dq0 = h->d_dq0; ra.geo = h->d_geo; ra.tab = h->tab;
    ra.e2f = h->d_e2f; ra.perm = h->d_perm; ra.dUH = dUH; ra.dQ = dQ; ra.dU = dU;
    prof_begin(h, HDG_K_RECOVER);
    k_recover_r<C, float, 256><<<(unsigned)h->E, 256, 0, h->stream>>>(mixed_regions(h), ra);
    prof_end(h);
    HDG_CK(cudaGetLastError());
    return HDG_OK;
}

#define HDG_INSTANTIATE_MIXED(D, P)                                            \
    template int run_linearize_mixed<D, P>(hdg_ctx*, const LinArgs&);          \
    template int run_recover_mixed<D, P>(hdg_ctx*, const double*, double*, double*);

}  // namespace hdg

namespace hdg {

// ----------------------------------------------------------------------------
// Schur product on the 5th-generation tensor cores: S^K = Dt - W Z per element,
// tcgen05.mma kind::tf32 with FP32 accumulation in tensor memory.  W rows and Z
// columns are staged by the CTA's threads into shared memory in the canonical
// K-major layout without swizzle (8-row x 16-byte core matrices; K-adjacent
// cores 128 B apart, 8-row groups KC/4 x 128 B apart).  SPLIT3 selects 3xTF32:
// x = hi + lo with hi = tf32(x), lo = tf32(x - hi), and W Z ~ Wh Zh + Wh Zl + Wl Zh.
// One CTA (4 warps) per (element, 128-row tile, column tile).  Waits on the
// MMA completion barrier are bounded; on timeout the CTA latches status bit 4,
// waits once more (bounded) and frees its tensor memory.
// ----------------------------------------------------------------------------
template <class C>
struct SchurTC {
    static constexpr int NT = C::NT, NU = C::NU;
    static constexpr int MT = 128, KC = 32;
    static constexpr int NNT = (NT + 127) / 128;                          // column tiles (<= 128 TMEM columns each)
    static constexpr int NTN = (((NT + NNT - 1) / NNT) + 15) / 16 * 16;   // columns per tile (mult. of 16)
    static constexpr int NMT = (NT + MT - 1) / MT;                        // row tiles
    static constexpr int TCOLS = NTN <= 32 ? 32 : NTN <= 64 ? 64 : NTN <= 128 ? 128 : 256;
    static_assert(NTN <= 256, "column tile too wide");
    static constexpr int THREADS = 256;
    static constexpr int WRS = KC + 4;                                    // raw W row stride (floats)
    __host__ __device__ static constexpr int tile_floats(int rows) { return rows * KC; }
    __host__ __device__ static constexpr int raw_floats() { return MT * WRS + KC * NTN; }
    __host__ __device__ static constexpr int smem_bytes(bool split3) {
        return (split3 ? 2 : 1) * (tile_floats(MT) + tile_floats(NTN)) * 4 + raw_floats() * 4 + 64;
    }
};



__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" :: "r"(smem_u32(dst)), "l"(src), "r"(src_bytes));
}

// One CTA (8 warps) per (element, 128-row tile, column tile).  The raw FP32 tiles of
// the next K chunk (W rows, Z rows) are copied into shared memory asynchronously
// (cp.async) while the tensor cores run the current chunk; the threads then split
// them into TF32 hi (/ lo) parts and store them in the core-matrix layout, rows
// fastest so that the 16-byte stores of a quarter warp are contiguous.
template <class C, bool SPLIT3>
__global__ void __launch_bounds__(SchurTC<C>::THREADS) k_schur_tc(Regions<float> R, int64_t e0, int32_t* status) {
    using S = SchurTC<C>;
    constexpr int NT = S::NT, NU = S::NU, MT = S::MT, KC = S::KC, NTN = S::NTN, TH = S::THREADS, WRS = S::WRS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t bid = blockIdx.x;
    const int nt = (int)(bid % S::NNT), mt = (int)((bid / S::NNT) % S::NMT);
    const int64_t el = bid / (S::NNT * S::NMT), e = e0 + el;
    const int m0 = mt * MT, n0 = nt * NTN;
    const float* W = R.a21 + el * R.a21_es;
    const float* Z = R.a12 + e * R.a12_es;
    float* Dm = R.a22 + el * R.a22_es;
    const int64_t sw = R.a21_rs, sz = R.a12_rs, sd = R.a22_rs;
    extern __shared__ __align__(1024) unsigned char smraw[];
    float* Ah = reinterpret_cast<float*>(smraw);
    float* Bh = Ah + S::tile_floats(MT);
    float* Al = Bh + S::tile_floats(NTN);
    float* Bl = Al + S::tile_floats(MT);
    float* Wr = (SPLIT3 ? Bl + S::tile_floats(NTN) : Al);       // [MT][WRS] raw W of the next chunk
    float* Zr = Wr + MT * WRS;                                  // [KC][NTN] raw Z
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smraw + S::smem_bytes(SPLIT3) - 64);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);

    auto prefetch = [&](int k0) {
        for (int it = tid; it < MT * KC; it += TH) {
            const int r = it / KC, k = it - r * KC;
            const bool in = m0 + r < NT && k0 + k < NU;
            cp_async4(Wr + r * WRS + k, in ? (const void*)(W + (m0 + r) * sw + k0 + k) : (const void*)W, in ? 4 : 0);
        }
        for (int it = tid; it < KC * NTN; it += TH) {
            const int k = it / NTN, n = it - k * NTN;
            const bool in = k0 + k < NU && n0 + n < NT;
            cp_async4(Zr + k * NTN + n, in ? (const void*)(Z + (k0 + k) * sz + n0 + n) : (const void*)Z, in ? 4 : 0);
        }
        asm volatile("cp.async.commit_group;");
    };
    prefetch(0);

    // right-hand side of this row tile: Rh -= W z (FP64), done by the first column tile
    if (nt == 0) {
        const double* z = R.rt + e * R.rt_es;
        double* rb = R.rb + el * R.rb_es;
        const int r = m0 + tid;
        if (tid < MT && r < NT) {
            double s = rb[r * R.rb_rs];
            for (int k = 0; k < NU; ++k) s -= (double)W[r * sw + k] * z[k * R.rt_rs];
            rb[r * R.rb_rs] = s;
        }
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(tslot)),
                     "r"(S::TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NTN >> 3) << 17) | ((uint32_t)(MT >> 4) << 24);
    const uint32_t bar = smem_u32(mbar);
    uint32_t phase = 0;
    bool ok = true, pending = false;
    for (int k0 = 0; k0 < NU; k0 += KC) {
        asm volatile("cp.async.wait_group 0;");
        if (pending) {                                          // the previous batch still reads the tiles
            if (!mbar_wait_bounded(bar, phase, 1 << 24)) {
                ok = false;
                if (tid == 0) atomicOr(status, 4);
                mbar_wait_bounded(bar, phase, 1 << 24);
            }
            phase ^= 1;
            pending = false;
        }
        if (__syncthreads_or(ok ? 0 : 1)) {                     // raw tiles visible, operand tiles free
            ok = false;
            break;
        }
        // item = (row, 4-wide K group q) -> one 16-byte core-matrix row; rows fastest
        for (int it = tid; it < MT * (KC / 4); it += TH) {
            const int r = it % MT, q = it / MT;
            const float4 v = *reinterpret_cast<const float4*>(Wr + r * WRS + q * 4);
            const int off = ((r >> 3) * (KC / 4) + q) * 32 + (r & 7) * 4;    // floats
            float4 hi = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
            *reinterpret_cast<float4*>(Ah + off) = hi;
            if (SPLIT3)
                *reinterpret_cast<float4*>(Al + off) =
                    make_float4(tf32_round(v.x - hi.x), tf32_round(v.y - hi.y), tf32_round(v.z - hi.z), tf32_round(v.w - hi.w));
        }
        for (int it = tid; it < NTN * (KC / 4); it += TH) {
            const int n = it % NTN, q = it / NTN;
            const float4 v = make_float4(Zr[(q * 4 + 0) * NTN + n], Zr[(q * 4 + 1) * NTN + n], Zr[(q * 4 + 2) * NTN + n],
                                         Zr[(q * 4 + 3) * NTN + n]);
            const int off = ((n >> 3) * (KC / 4) + q) * 32 + (n & 7) * 4;
            float4 hi = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
            *reinterpret_cast<float4*>(Bh + off) = hi;
            if (SPLIT3)
                *reinterpret_cast<float4*>(Bl + off) =
                    make_float4(tf32_round(v.x - hi.x), tf32_round(v.y - hi.y), tf32_round(v.z - hi.z), tf32_round(v.w - hi.w));
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();                                        // tiles staged, raw tiles consumed
        if (k0 + KC < NU) prefetch(k0 + KC);                    // next chunk under this chunk's MMAs
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int nsteps = (min(KC, NU - k0) + 7) / 8;
            for (int st = 0; st < nsteps; ++st) {
                const uint32_t off = st * 256;
                const uint64_t ah = umma_desc(smem_u32(Ah) + off, 128, (KC / 4) * 128);
                const uint64_t bh = umma_desc(smem_u32(Bh) + off, 128, (KC / 4) * 128);
                uint32_t acc = (k0 > 0 || st > 0) ? 1u : 0u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                             :: "r"(tmem), "l"(ah), "l"(bh), "r"(idesc), "r"(acc));
                if (SPLIT3) {
                    const uint64_t al = umma_desc(smem_u32(Al) + off, 128, (KC / 4) * 128);
                    const uint64_t bl = umma_desc(smem_u32(Bl) + off, 128, (KC / 4) * 128);
                    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;"
                                 :: "r"(tmem), "l"(ah), "l"(bl), "r"(idesc));
                    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;"
                                 :: "r"(tmem), "l"(al), "l"(bh), "r"(idesc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar));
        }
        pending = true;
    }
    asm volatile("cp.async.wait_group 0;");
    if (pending && ok) {
        if (!mbar_wait_bounded(bar, phase, 1 << 24)) {
            ok = false;
            if (tid == 0) atomicOr(status, 4);
            mbar_wait_bounded(bar, phase, 1 << 24);
        }
        phase ^= 1;
    }
    ok = !__syncthreads_or(ok ? 0 : 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        // warp w reads lanes 32 (w % 4) .. + 31 and the column half w / 4 of the tile
        const int lg = warp & 3, half = warp >> 2;
        const int r = m0 + lg * 32 + lane;
        constexpr int HC = ((NTN / 2) + 15) / 16 * 16;          // columns per half, in chunks of 16
#pragma unroll 1
        for (int c0 = half * HC; c0 < min(NTN, (half + 1) * HC); c0 += 16) {
            uint32_t v[16];
            const uint32_t addr = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                           "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                         : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (r < NT) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = n0 + c0 + j;
                    if (c0 + j < NTN && c < NT) Dm[r * sd + c] -= __uint_as_float(v[j]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(S::TCOLS));
}

template <class C>
struct BlkTC {
    static constexpr int NCB = C::NP + C::NF * C::NFP;
    static constexpr int MR = C::M * C::M * NCB;
    static constexpr int MT = 128, KC = 16;   // 16-wide chunks keep 4-5 CTAs (32-40 warps) per SM
    static constexpr int NMT = (MR + MT - 1) / MT;
    static constexpr int K = C::D * C::NQ;
    static constexpr int CPD = (C::NQ + KC - 1) / KC;                     // chunks per direction
    static constexpr int NCH = C::D * CPD;                                // chunks in all
    static constexpr int NTN = (C::NP + 15) / 16 * 16;
    static constexpr int TCOLS = NTN <= 32 ? 32 : NTN <= 64 ? 64 : 128;
    static constexpr int THREADS = 256;
    static_assert(THREADS == 2 * MT, "a thread forms one row for two K quads");
    static constexpr int STAGE = 2 * (MT * KC + NTN * KC);                // floats of one stage (hi and lo)
    static constexpr int MINB = NTN <= 32 ? 5 : 3;                        // resident CTAs (registers, stages)
    static_assert(NTN <= 128, "N tile too wide");
    __host__ __device__ static constexpr int smem_bytes() { return 2 * STAGE * 4 + 64; }
};

// Volume contraction of the mixed form on the tensor cores: Out[(a, b, c)][i] =
// sum_k G_ab[k][c] dphi[k][i] per element, 3xTF32 with FP32 accumulation in TMEM.
// 8 warps per (element, 128-row tile); the operand tiles are double-buffered so that
// the threads generate chunk c + 1 (rows fastest: a quarter warp's 16-byte stores are
// contiguous) while the tensor cores run chunk c.
template <class C>
__global__ void __launch_bounds__(BlkTC<C>::THREADS, BlkTC<C>::MINB) k_blocks_tc(BlkArgs<float> A, int32_t* status) {
    using S = BlkTC<C>;
    constexpr int D = C::D, M = C::M, NP = C::NP, NQ = C::NQ, NFP = C::NFP, NCOEF = C::NCOEF;
    constexpr int NCB = S::NCB, MR = S::MR, MT = S::MT, KC = S::KC, NTN = S::NTN, TH = S::THREADS;
    constexpr int GEO = Geo<D>::N;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t bid = blockIdx.x;
    const int mt = (int)(bid % S::NMT);
    const int64_t el = bid / S::NMT, e = A.e0 + el;
    const int m0 = mt * MT;
    const DeviceTables& T = A.tab;
    const float* cfe = reinterpret_cast<const float*>(A.vcoef) + (size_t)el * M * M * D * NCOEF * NQ;
    extern __shared__ __align__(1024) unsigned char smraw[];
    float* stage0 = reinterpret_cast<float*>(smraw);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smraw + S::smem_bytes() - 64);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);

    // Chunks run over one direction and 16 consecutive points each (every
    // direction's points padded to whole chunks), so that a chunk needs no
    // division per entry; thread tid forms row tid % 128 (decoded once) for the
    // K quads tid / 128 and tid / 128 + 2, each quad's loads issued before they are used.
    const int rl = tid & (MT - 1), r0 = m0 + rl;
    const bool live = r0 < MR;
    const int rab = live ? r0 / NCB : 0, rc = live ? r0 - rab * NCB : 0;
    const bool vol = rc < NP;
    const int rf = vol ? 0 : (rc - NP) / NFP, rlf = vol ? 0 : rc - NP - rf * NFP;
    const float* rcf = cfe + (size_t)rab * D * NCOEF * NQ;

    // operand tiles of chunk ci into stage buffer sb (Ah | Bh | Al | Bl)
    auto generate = [&](int ci, float* sb) {
        float* Ah = sb;
        float* Bh = Ah + MT * KC;
        float* Al = Bh + NTN * KC;
        float* Bl = Al + MT * KC;
        const int dir = ci / S::CPD, g0 = (ci - dir * S::CPD) * KC;
        const float* cc = rcf + (size_t)dir * NCOEF * NQ;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {                  // one K quad at a time: its loads in flight together
            const int q = (tid >> 7) + 2 * h;
            float v[4];
            if (vol) {
                float c0[4], t0[4], cr[4][D], tr[4][D];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int g = min(g0 + 4 * q + u, NQ - 1);
                    c0[u] = cc[g];
                    t0[u] = T.fphi[g * NP + rc];
#pragma unroll
                    for (int r2 = 0; r2 < D; ++r2) {
                        cr[u][r2] = cc[(1 + r2) * NQ + g];
                        tr[u][r2] = T.fpsi[((size_t)r2 * NQ + g) * NP + rc];
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float x = c0[u] * t0[u];
#pragma unroll
                    for (int r2 = 0; r2 < D; ++r2) x = fmaf(-cr[u][r2], tr[u][r2], x);
                    v[u] = x;
                }
            } else {
                float c1[4], t1[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int g = min(g0 + 4 * q + u, NQ - 1);
                    c1[u] = cc[(1 + D + rf) * NQ + g];
                    t1[u] = T.ftheta[((size_t)rf * NQ + g) * NFP + rlf];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = c1[u] * t1[u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (!live || g0 + 4 * q + u >= NQ) v[u] = 0.f;
            const int off = ((rl >> 3) * (KC / 4) + q) * 32 + (rl & 7) * 4;
            const float4 hi = make_float4(tf32_round(v[0]), tf32_round(v[1]), tf32_round(v[2]), tf32_round(v[3]));
            *reinterpret_cast<float4*>(Ah + off) = hi;
            *reinterpret_cast<float4*>(Al + off) = make_float4(tf32_round(v[0] - hi.x), tf32_round(v[1] - hi.y),
                                                               tf32_round(v[2] - hi.z), tf32_round(v[3] - hi.w));
        }
        for (int it = tid; it < NTN * (KC / 4); it += TH) {
            const int n = it % NTN, q = it / NTN;
            float w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int g = g0 + q * 4 + u;
                w[u] = (n < NP && g < NQ) ? T.fdphi[((size_t)dir * NQ + g) * NP + n] : 0.f;
            }
            const int off = ((n >> 3) * (KC / 4) + q) * 32 + (n & 7) * 4;
            const float4 hi = make_float4(tf32_round(w[0]), tf32_round(w[1]), tf32_round(w[2]), tf32_round(w[3]));
            *reinterpret_cast<float4*>(Bh + off) = hi;
            *reinterpret_cast<float4*>(Bl + off) = make_float4(tf32_round(w[0] - hi.x), tf32_round(w[1] - hi.y),
                                                               tf32_round(w[2] - hi.z), tf32_round(w[3] - hi.w));
        }
        asm volatile("fence.proxy.async.shared::cta;");
    };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(tslot)),
                     "r"(S::TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar + 1)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    generate(0, stage0);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NTN >> 3) << 17) | ((uint32_t)(MT >> 4) << 24);
    // one barrier per stage buffer: the batch that reads buffer s commits to barrier s, and
    // is waited for before buffer s is written again, so no barrier runs two phases ahead
    uint32_t phase = 0u, pending = 0u;                          // bit s: barrier s
    bool ok = true;
    auto wait_stage = [&](int sb) {
        if (!((pending >> sb) & 1u)) return;
        const uint32_t bar = smem_u32(mbar + sb), par = (phase >> sb) & 1u;
        if (!mbar_wait_bounded(bar, par, 1 << 24)) {
            ok = false;
            if (tid == 0) atomicOr(status, 4);
            mbar_wait_bounded(bar, par, 1 << 24);
        }
        phase ^= 1u << sb;
        pending &= ~(1u << sb);
    };
    for (int ci = 0; ci < S::NCH; ++ci) {
        const int sbi = ci & 1;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const float* Ah = stage0 + sbi * S::STAGE;
            const float* Bh = Ah + MT * KC;
            const float* Al = Bh + NTN * KC;
            const float* Bl = Al + MT * KC;
            for (int s = 0; s < KC / 8; ++s) {
                const uint32_t off = s * 256;
                const uint64_t ah = umma_desc(smem_u32(Ah) + off, 128, (KC / 4) * 128);
                const uint64_t bh = umma_desc(smem_u32(Bh) + off, 128, (KC / 4) * 128);
                const uint64_t al = umma_desc(smem_u32(Al) + off, 128, (KC / 4) * 128);
                const uint64_t bl = umma_desc(smem_u32(Bl) + off, 128, (KC / 4) * 128);
                uint32_t acc = (ci > 0 || s > 0) ? 1u : 0u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                             :: "r"(tmem), "l"(ah), "l"(bh), "r"(idesc), "r"(acc));
                asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;"
                             :: "r"(tmem), "l"(ah), "l"(bl), "r"(idesc));
                asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;"
                             :: "r"(tmem), "l"(al), "l"(bh), "r"(idesc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(mbar + sbi)));
        }
        pending |= 1u << sbi;
        if (ci + 1 < S::NCH) {
            wait_stage(sbi ^ 1);                                 // the batch before this one read the other buffer
            if (__syncthreads_or(ok ? 0 : 1)) {
                ok = false;
                break;
            }
            generate(ci + 1, stage0 + (sbi ^ 1) * S::STAGE);
            __syncthreads();
        }
    }
    wait_stage(0);                                               // every batch completes before the epilogue
    wait_stage(1);
    ok = !__syncthreads_or(ok ? 0 : 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        // warp w reads lanes 32 (w % 4) .. + 31; warps 4..7 take the second half of the columns
        const int lg = warp & 3, half = warp >> 2;
        const int r = m0 + lg * 32 + lane;
        const int ab = r / NCB, c = r - ab * NCB, a = ab / M, b = ab - a * M;
        const double detJ = A.geo[e * GEO];
        double* A11 = A.R.a11 + e * A.R.a11_es;
        float* A12 = A.R.a12 + e * A.R.a12_es;
        constexpr int HC = ((NTN / 2) + 15) / 16 * 16;
#pragma unroll 1
        for (int c0 = half * HC; c0 < min(NTN, (half + 1) * HC); c0 += 16) {
            uint32_t v[16];
            const uint32_t addr = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                           "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                         : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (r < MR) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int i = c0 + j;
                    if (i >= NP) continue;
                    const float x = __uint_as_float(v[j]);
                    const int64_t row = a * NP + i;
                    if (c < NP) {
                        double w = (double)x;
                        if (a == b) w += detJ / A.a_ii * T.mhat[i * NP + c];
                        A11[row * A.R.a11_rs + b * NP + c] = w;
                    } else {
                        const int c2 = c - NP, f = c2 / NFP, l = c2 - f * NFP;
                        A12[row * A.R.a12_rs + (f * M + b) * NFP + l] = x;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(S::TCOLS));
}

}  // namespace hdg
