// One-level additive Schwarz preconditioner of the tetrahedral trace system on
// element-centred face patches (Sec. 3.3, eq. additive-schwarz):
//     M^{-1} = sum_r R_r^T S_r^{-1} R_r,   S_r = R_r S R_r^T,
// R_r the restriction to the trace unknowns of the four faces of element r
// (local face order, each face's block in its canonical order), no coarse
// space.  Patch sizes vary with the degrees of the element's faces (t = 60 to
// 300 for degrees 1..4).
//
// Set-up: one CTA per patch, taken from a cost-ordered work list by a
// persistent grid, gathers S_r from the assembled blocks into a row-major
// [t][LDA] matrix and factors it by LU with partial pivoting in the system's
// precision (FP64 system: FP64; mixed form: FP32), with the runtime-sized panel
// elimination of the linearization; the interchanges are then applied to the
// columns left of each panel, so that P S_r = L U, and P is stored as a gather
// map.  Apply: one CTA per patch gathers P R_r x, solves L U z = P R_r x by
// blocked substitution (32-row blocks: the off-diagonal part by warp dot
// products, the diagonal block by one warp with shuffles), and a second kernel
// sums the patch corrections of each face over its elements in ascending
// element order (bitwise reproducible).
#include <algorithm>
#include <cstring>

#include "solve.cuh"
#include "tet.h"
#include "tet_elim.cuh"

namespace hdg {
namespace tet {

constexpr int ASM_NB = 16;               // panel width of the patch LU
constexpr int TMAX = 4 * M * NFPMAX;     // largest patch (four degree-4 faces)
constexpr int ASM_SOLVE_THREADS = 128;

__device__ __forceinline__ int patch_face(const TetElem& d, int i) {
    int f = 0;
    while (f < 3 && i >= d.toff[f + 1]) ++f;
    return f;
}

template <class T>
__global__ void __launch_bounds__(NTH, 2) k_tet_asm_factor(const TetElem* __restrict__ el, const int32_t* order,
                                                           int64_t E, int32_t* next, const T* __restrict__ vals,
                                                           const int64_t* __restrict__ boff,
                                                           const int32_t* __restrict__ rowptr,
                                                           const int32_t* __restrict__ col,
                                                           const int64_t* __restrict__ aoff,
                                                           const int64_t* __restrict__ poff, T* lu, int32_t* perm,
                                                           int32_t* status) {
    extern __shared__ __align__(16) unsigned char asm_raw[];
    T* pan = reinterpret_cast<T*>(asm_raw);              // [TMAX][ASM_NB]
    T* ust = pan + TMAX * ASM_NB;                        // [ASM_NB][TCW]
    __shared__ int piv[ASM_NB];
    __shared__ int sflag;
    __shared__ int64_t s_e;
    __shared__ int32_t sblk[16];
    __shared__ int32_t sperm[TMAX];
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) {
            const int k = atomicAdd(next, 1);
            s_e = k < E ? order[k] : -1;
            sflag = 0;
        }
        __syncthreads();
        const int64_t e = s_e;
        if (e < 0) break;
        const TetElem& d = el[e];
        const int t = d.t, lda = (t + 3) & ~3;
        T* A = lu + aoff[e];
        int32_t* gp = perm + poff[e];
        if (tid < 16) {                                  // block (face fi, face fj) of S in row face fi
            const int fi = tid >> 2, fj = tid & 3;
            const int64_t Fi = d.face[fi], Fj = d.face[fj];
            int32_t b = -1;
            for (int32_t k = rowptr[Fi]; k < rowptr[Fi + 1]; ++k)
                if (col[k] == (int32_t)Fj) { b = k; break; }
            sblk[tid] = b;
        }
        __syncthreads();
        for (int idx = tid; idx < t * t; idx += NTH) {   // S_r, row-major
            const int j = idx / t, i = idx - j * t;
            const int fi = patch_face(d, i), fj = patch_face(d, j);
            const int32_t b = sblk[fi * 4 + fj];
            const int r = i - d.toff[fi], c = j - d.toff[fj];
            A[(size_t)i * lda + j] = b >= 0 ? vals[boff[b] + (int64_t)c * (M * d.nfp[fi]) + r] : T(0);
        }
        __syncthreads();
        bordered_elim<ASM_NB, T>(A, t, t, t, lda, pan, ust, piv, &sflag, gp);
        __syncthreads();
        // interchanges of each panel applied to the columns left of it, in panel order
        for (int k0 = ASM_NB; k0 < t; k0 += ASM_NB) {
            const int kb = min(ASM_NB, t - k0);
            for (int j = 0; j < kb; ++j) {
                const int pr = gp[k0 + j];
                if (pr != k0 + j) {
                    for (int c = tid; c < k0; c += NTH) {
                        T* x = A + (size_t)(k0 + j) * lda + c;
                        T* y = A + (size_t)pr * lda + c;
                        const T v = *x;
                        *x = *y;
                        *y = v;
                    }
                }
                __syncthreads();
            }
        }
        if (tid == 0) {                                  // P as a gather map: (P b)_i = b_perm[i]
            for (int i = 0; i < t; ++i) sperm[i] = i;
            for (int k = 0; k < t; ++k) {
                const int pr = gp[k];
                const int v = sperm[k];
                sperm[k] = sperm[pr];
                sperm[pr] = v;
            }
            if (sflag) atomicOr(status, sflag);
        }
        __syncthreads();
        for (int i = tid; i < t; i += NTH) gp[i] = sperm[i];
        __syncthreads();
    }
}

template <class T>
__device__ __forceinline__ T warp_sum(T s) {
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    return s;
}

// z_r = S_r^{-1} R_r x = U^{-1} L^{-1} P R_r x for every patch, in the factors' precision
template <class T>
__global__ void __launch_bounds__(ASM_SOLVE_THREADS) k_tet_asm_solve(const TetElem* __restrict__ el,
                                                                     const T* __restrict__ lu,
                                                                     const int64_t* __restrict__ aoff,
                                                                     const int32_t* __restrict__ perm,
                                                                     const int64_t* __restrict__ poff,
                                                                     const double* __restrict__ x, double* z) {
    __shared__ T y[TMAX];
    __shared__ T D[32][33];
    __shared__ T part[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = ASM_SOLVE_THREADS / 32;
    const int64_t e = blockIdx.x;
    const TetElem& d = el[e];
    const int t = d.t, lda = (t + 3) & ~3;
    const T* A = lu + aoff[e];
    const int32_t* pm = perm + poff[e];
    for (int i = tid; i < t; i += ASM_SOLVE_THREADS) {
        const int s = pm[i], f = patch_face(d, s);
        y[i] = (T)x[d.hoff[f] + (s - d.toff[f])];
    }
    __syncthreads();
    // forward substitution with the unit lower factor
    for (int b0 = 0; b0 < t; b0 += 32) {
        const int nb = min(32, t - b0);
        for (int rr = warp; rr < nb; rr += NW) {
            const T* row = A + (size_t)(b0 + rr) * lda;
            T s = T(0);
            for (int k = lane; k < b0; k += 32) s = fma(row[k], y[k], s);
            s = warp_sum(s);
            if (lane == 0) part[rr] = s;
        }
        for (int idx = tid; idx < nb * 32; idx += ASM_SOLVE_THREADS) {
            const int r = idx >> 5, c = idx & 31;
            if (c < nb) D[r][c] = A[(size_t)(b0 + r) * lda + b0 + c];
        }
        __syncthreads();
        if (warp == 0) {
            T v = lane < nb ? y[b0 + lane] - part[lane] : T(0);
            for (int k = 0; k < nb; ++k) {
                const T yk = __shfl_sync(0xffffffffu, v, k);
                if (lane > k && lane < nb) v = fma(-D[lane][k], yk, v);
            }
            if (lane < nb) y[b0 + lane] = v;
        }
        __syncthreads();
    }
    // back substitution with the upper factor
    for (int b1 = t; b1 > 0; b1 -= 32) {
        const int b0 = max(0, b1 - 32), nb = b1 - b0;
        for (int rr = warp; rr < nb; rr += NW) {
            const T* row = A + (size_t)(b0 + rr) * lda;
            T s = T(0);
            for (int k = b1 + lane; k < t; k += 32) s = fma(row[k], y[k], s);
            s = warp_sum(s);
            if (lane == 0) part[rr] = s;
        }
        for (int idx = tid; idx < nb * 32; idx += ASM_SOLVE_THREADS) {
            const int r = idx >> 5, c = idx & 31;
            if (c < nb) D[r][c] = A[(size_t)(b0 + r) * lda + b0 + c];
        }
        __syncthreads();
        if (warp == 0) {
            T v = lane < nb ? y[b0 + lane] - part[lane] : T(0);
            for (int k = nb - 1; k >= 0; --k) {
                if (lane == k) {
                    T dk = D[k][k];
                    if (dk == T(0) || !isfinite(dk)) dk = T(1);   // flagged at set-up
                    v = v / dk;
                }
                const T xk = __shfl_sync(0xffffffffu, v, k);
                if (lane < k) v = fma(-D[lane][k], xk, v);
            }
            if (lane < nb) y[b0 + lane] = v;
        }
        __syncthreads();
    }
    double* zr = z + poff[e];
    for (int i = tid; i < t; i += ASM_SOLVE_THREADS) zr[i] = (double)y[i];
}

// y_F = sum over the elements K of face F (ascending id) of the patch correction of K on F
__global__ void k_tet_asm_sum(const TetElem* __restrict__ el, const int64_t* __restrict__ hoff,
                              const int32_t* __restrict__ f2e, const int32_t* __restrict__ f2lf,
                              const int64_t* __restrict__ poff, const double* __restrict__ z, int64_t F, double* y) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t Fr = wid; Fr < F; Fr += nw) {
        int e0 = f2e[2 * Fr], e1 = f2e[2 * Fr + 1], l0 = f2lf[2 * Fr], l1 = f2lf[2 * Fr + 1];
        if (e1 >= 0 && e1 < e0) { int tt = e0; e0 = e1; e1 = tt; tt = l0; l0 = l1; l1 = tt; }
        const int bs = (int)(hoff[Fr + 1] - hoff[Fr]);
        const double* z0 = z + poff[e0] + el[e0].toff[l0];
        const double* z1 = e1 >= 0 ? z + poff[e1] + el[e1].toff[l1] : nullptr;
        for (int r = lane; r < bs; r += 32) {
            double v = z0[r];
            if (z1) v += z1[r];
            y[hoff[Fr] + r] = v;
        }
    }
}

namespace {

template <class T>
int asm_alloc(hdg_ctx* h, T** out, size_t count) {
    void* p = nullptr;
    const cudaError_t e = cudaMalloc(&p, std::max<size_t>(1, count) * sizeof(T));
    if (e != cudaSuccess) {
        h->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? HDG_ENOMEM : HDG_ECUDA;
    }
    h->allocs.push_back(p);
    h->device_bytes += (int64_t)(std::max<size_t>(1, count) * sizeof(T));
    *out = static_cast<T*>(p);
    return HDG_OK;
}

#define ASM_CK(call)                                                                   \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            h->err = std::string(#call) + ": " + cudaGetErrorString(e_);               \
            return HDG_ECUDA;                                                          \
        }                                                                              \
    } while (0)

}  // namespace

int asm_setup(hdg_ctx* h) {
    Ctx* c = h->tet;
    if (!c->have_system) { h->err = "no assembled trace system"; return HDG_EINVAL; }
    int rc;
    if (!c->d_aoff) {
        std::vector<int64_t> aoff(c->E + 1), poff(c->E + 1);
        aoff[0] = poff[0] = 0;
        for (int64_t e = 0; e < c->E; ++e) {
            const int t = c->el[e].t;
            if (t > TMAX) { h->err = "patch larger than four degree-4 faces"; return HDG_EINVAL; }
            aoff[e + 1] = aoff[e] + (int64_t)t * ((t + 3) & ~3);
            poff[e + 1] = poff[e] + t;
        }
        c->n_asm = aoff[c->E];
        c->n_patch = poff[c->E];
        if ((rc = asm_alloc(h, &c->d_aoff, aoff.size()))) return rc;
        if ((rc = asm_alloc(h, &c->d_poff, poff.size()))) return rc;
        ASM_CK(cudaMemcpy(c->d_aoff, aoff.data(), sizeof(int64_t) * aoff.size(), cudaMemcpyHostToDevice));
        ASM_CK(cudaMemcpy(c->d_poff, poff.data(), sizeof(int64_t) * poff.size(), cudaMemcpyHostToDevice));
        if ((rc = asm_alloc(h, &c->d_asmperm, (size_t)c->n_patch))) return rc;
        if ((rc = asm_alloc(h, &c->d_asmz, (size_t)c->n_patch))) return rc;
        if ((rc = asm_alloc(h, &c->d_asmnext, 1))) return rc;
        const size_t sm64 = sizeof(double) * ((size_t)TMAX * ASM_NB + ASM_NB * TCW);
        const size_t sm32 = sizeof(float) * ((size_t)TMAX * ASM_NB + ASM_NB * TCW);
        ASM_CK(cudaFuncSetAttribute(k_tet_asm_factor<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm64));
        ASM_CK(cudaFuncSetAttribute(k_tet_asm_factor<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm32));
    }
    const bool mixed = c->sys_prec != HDG_PREC_FP64;
    if (!mixed && !c->d_asm && (rc = asm_alloc(h, &c->d_asm, (size_t)c->n_asm))) return rc;
    if (mixed && !c->d_asm32 && (rc = asm_alloc(h, &c->d_asm32, (size_t)c->n_asm))) return rc;
    int dev = 0, nsm = 0;
    ASM_CK(cudaGetDevice(&dev));
    ASM_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const unsigned grid = (unsigned)std::min<int64_t>(c->E, 2LL * nsm);
    cudaStream_t st = h->stream;
    ASM_CK(cudaMemsetAsync(c->d_asmnext, 0, sizeof(int32_t), st));
    if (!mixed) {
        const size_t sm = sizeof(double) * ((size_t)TMAX * ASM_NB + ASM_NB * TCW);
        k_tet_asm_factor<double><<<grid, NTH, sm, st>>>(c->d_el, c->d_order, c->E, c->d_asmnext, c->d_vals,
                                                       c->d_boff, c->d_rowptr, c->d_col, c->d_aoff, c->d_poff,
                                                       c->d_asm, c->d_asmperm, h->d_status);
    } else {
        const size_t sm = sizeof(float) * ((size_t)TMAX * ASM_NB + ASM_NB * TCW);
        k_tet_asm_factor<float><<<grid, NTH, sm, st>>>(c->d_el, c->d_order, c->E, c->d_asmnext, c->d_vals32,
                                                      c->d_boff, c->d_rowptr, c->d_col, c->d_aoff, c->d_poff,
                                                      c->d_asm32, c->d_asmperm, h->d_status);
    }
    ASM_CK(cudaGetLastError());
    c->asm_prec = mixed ? HDG_PREC_MIXED : HDG_PREC_FP64;
    c->asm_ready = true;
    return HDG_OK;
}

int asm_apply(hdg_ctx* h, const double* x, double* y) {
    Ctx* c = h->tet;
    cudaStream_t st = h->stream;
    if (c->asm_prec == HDG_PREC_FP64)
        k_tet_asm_solve<double><<<(unsigned)c->E, ASM_SOLVE_THREADS, 0, st>>>(c->d_el, c->d_asm, c->d_aoff,
                                                                             c->d_asmperm, c->d_poff, x, c->d_asmz);
    else
        k_tet_asm_solve<float><<<(unsigned)c->E, ASM_SOLVE_THREADS, 0, st>>>(c->d_el, c->d_asm32, c->d_aoff,
                                                                            c->d_asmperm, c->d_poff, x, c->d_asmz);
    const unsigned gf = (unsigned)std::min<int64_t>(65535, (c->F + 7) / 8);
    k_tet_asm_sum<<<gf, 256, 0, st>>>(c->d_el, c->d_hoff, c->d_f2e, c->d_f2lf, c->d_poff, c->d_asmz, c->F, y);
    ASM_CK(cudaGetLastError());
    return HDG_OK;
}

}  // namespace tet
}  // namespace hdg
