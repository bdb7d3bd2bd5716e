// Runtime-sized dense elimination shared by the tetrahedral kernels: the
// per-element bordered elimination of the linearization (interior LU with
// partial pivoting, Schur complement of the trace rows) and the LU of the
// additive-Schwarz patch matrices.  One CTA of NTH threads per matrix.
#pragma once

#include <climits>

namespace hdg {
namespace tet {

constexpr int NTH = 256;                  // threads of the tetrahedral kernels
constexpr int TCW = 64;                   // elimination column tile

// runtime-sized tile of the trailing update A22 -= L21 U12 (rows rb + ty + 16 ii,
// columns ct + tx + 16 jj)
template <int NII, int NJJ, int NB, class T, class RowP>
__device__ __forceinline__ void trail_tile_rt(RowP rowp, const T* pan, const T* ust, int rb, int ct, int k0,
                                              int kb, int tx, int ty, int NR, int NC) {
    T acc[NII][NJJ];
    T* rp[NII];
#pragma unroll
    for (int ii = 0; ii < NII; ++ii) {
        const int r = rb + ty + 16 * ii;
        rp[ii] = (r < NR) ? rowp(r) : nullptr;
#pragma unroll
        for (int jj = 0; jj < NJJ; ++jj) {
            const int c = ct + tx + 16 * jj;
            acc[ii][jj] = (rp[ii] && c < NC) ? rp[ii][c] : T(0);
        }
    }
    const T* lp = pan + (size_t)(rb + ty - k0) * NB;
    for (int j = 0; j < kb; ++j) {
        T lv[NII], uv[NJJ];
#pragma unroll
        for (int ii = 0; ii < NII; ++ii) lv[ii] = (rb + ty + 16 * ii < NR) ? lp[16 * ii * NB + j] : T(0);
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
            const int c = ct + tx + 16 * jj;
            if (c < NC) rp[ii][c] = acc[ii][jj];
        }
    }
}

// Bordered elimination of the row-major matrix Mx [NR][LD] (columns NC; the
// linearization passes NC = NR + 1): LU with partial pivoting in the top NU rows
// (largest magnitude, lowest row on ties), panel by panel (NB columns); each
// panel's interchanges are applied to the panel and to the columns right of it,
// the rows below NU are eliminated, so that the bottom-right block becomes
// S = Dt - Ct At^{-1} Bt and the last column Rh - Ct At^{-1} Rt.  Columns left
// of a panel keep their rows (the L factor is stored as eliminated); gpiv, when
// not NULL, receives the pivot row of every eliminated column (global index),
// from which a caller can apply the interchanges to those columns afterwards.
// pan: [NR][NB], ust: [NB][TCW] shared memory; piv: [NB] shared.
template <int NB, class T>
__device__ void bordered_elim(T* Mx, int NU, int NR, int NC, int LD, T* pan, T* ust, int* piv, int* sflag,
                              int* gpiv = nullptr) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto rowp = [&](int r) -> T* { return Mx + (size_t)r * LD; };
    for (int k0 = 0; k0 < NU; k0 += NB) {
        const int kb = min(NB, NU - k0), nrows = NR - k0, ntop = NU - k0;
#pragma unroll 1
        for (int idx = tid; idx < nrows * kb; idx += NTH) {
            const int rr = idx / kb, c = idx - rr * kb;
            pan[rr * NB + c] = rowp(k0 + rr)[k0 + c];
        }
        __syncthreads();
        for (int j = 0; j < kb; ++j) {
            if (warp == 0) {
                T bv = T(-1);
                int bi = INT_MAX;
#pragma unroll 1
                for (int rr = j + lane; rr < ntop; rr += 32) {
                    const T v = fabs(pan[rr * NB + j]);
                    if (v > bv) { bv = v; bi = rr; }
                }
                for (int off = 16; off > 0; off >>= 1) {
                    const T ov = __shfl_down_sync(0xffffffffu, bv, off);
                    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
                    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
                }
                int pr = __shfl_sync(0xffffffffu, bi, 0);
                if (pr == INT_MAX) {
                    pr = j;
                    if (lane == 0) *sflag |= 2;
                }
                if (lane < kb && pr != j) {
                    const T t = pan[j * NB + lane];
                    pan[j * NB + lane] = pan[pr * NB + lane];
                    pan[pr * NB + lane] = t;
                }
                if (lane == 0) {
                    piv[j] = pr;
                    if (gpiv) gpiv[k0 + j] = k0 + pr;
                }
            }
            __syncthreads();
            T pv = pan[j * NB + j];
            if (pv == T(0) || !isfinite(pv)) {
                if (tid == 0) *sflag |= (pv == T(0)) ? 1 : 2;
                pv = T(1);
            }
            const T inv = T(1) / pv;
#pragma unroll 1
            for (int rr = j + 1 + tid; rr < nrows; rr += NTH) {
                const T l = pan[rr * NB + j] * inv;
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
        const int c0 = k0 + kb;
#pragma unroll 1
        for (int c = c0 + tid; c < NC; c += NTH) {
            for (int j = 0; j < kb; ++j) {
                const int pr = piv[j];
                if (pr != j) {
                    T* x = rowp(k0 + j) + c;
                    T* y = rowp(k0 + pr) + c;
                    const T t = *x;
                    *x = *y;
                    *y = t;
                }
            }
            T xv[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                if (j < kb) {
                    T s = rowp(k0 + j)[c];
#pragma unroll
                    for (int i = 0; i < NB; ++i)
                        if (i < j) s = fma(-pan[j * NB + i], xv[i], s);
                    xv[j] = s;
                    rowp(k0 + j)[c] = s;
                }
            }
        }
        __syncthreads();
        const int tx = tid & 15, ty = tid >> 4;
#pragma unroll 1
        for (int ct = c0; ct < NC; ct += TCW) {
            for (int idx = tid; idx < kb * TCW; idx += NTH) {
                const int j = idx / TCW, cc = idx - j * TCW;
                ust[j * TCW + cc] = (ct + cc < NC) ? rowp(k0 + j)[ct + cc] : T(0);
            }
            __syncthreads();
            int njj = 0;
            while (njj < 4 && ct + 16 * njj < NC) ++njj;
#pragma unroll 1
            for (int rb = c0; rb < NR; rb += 64) {
                int nii = 0;
                while (nii < 4 && rb + 16 * nii < NR) ++nii;
                switch (nii * 4 + njj - 5) {
#define HDG_TT(I, J) \
    case (I) * 4 + (J) - 5: trail_tile_rt<I, J, NB, T>(rowp, pan, ust, rb, ct, k0, kb, tx, ty, NR, NC); break;
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



}  // namespace tet
}  // namespace hdg
