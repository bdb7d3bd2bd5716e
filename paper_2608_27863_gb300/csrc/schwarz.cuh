// One-level additive Schwarz preconditioner on element-centred face patches
// (Sec. 3.3, eq. additive-schwarz):  M^{-1} = sum_r R_r^T S_r^{-1} R_r, where
// R_r restricts a trace vector to the nf faces of element r and
// S_r = R_r S R_r^T is the t x t patch of the assembled trace operator.
//
// Setup: one CTA per element gathers S_r from the block-sparse values (the
// (f, g) blocks of an element are listed in the skeleton's blk table) and
// factors it in place, P S_r = L U with partial pivoting (blocked, NB-column
// panels in shared memory, LAPACK-style full-row interchanges).  The factors
// are kept in the system's storage type: FP64 for the FP64 form, FP32 for the
// mixed form, where the preconditioner only needs to be a good approximation.
// Apply: one CTA per element solves its patch in the storage precision (blocked
// triangular solves with the 32 x 32 diagonal blocks pre-inverted at setup,
// one dot product per row and thread for the off-diagonal blocks), writes z_r, and a
// face kernel sums the (at most two) patch corrections of each face in a
// fixed order, so the result is bitwise reproducible.
#pragma once

namespace hdg {

template <class C>
struct AsmShape {
    static constexpr int N = C::NT;                 // patch unknowns
    static constexpr int LDA = (C::NT + 3) & ~3;    // padded row stride
};

template <class T, int NB>
constexpr int asm_factor_smem_bytes(int n) { return (n * NB + NB * 64) * (int)sizeof(T); }

template <class C, class T, int NB, int NTH>
__global__ void __launch_bounds__(NTH) k_asm_factor(const T* __restrict__ vals, const int32_t* __restrict__ blk,
                                                    T* __restrict__ lu, int32_t* __restrict__ piv_out,
                                                    int32_t* status) {
    constexpr int N = AsmShape<C>::N, LDA = AsmShape<C>::LDA, NF = C::NF, BS = C::BS;
    static_assert(NTH == 256, "trailing-update layout assumes 256 threads");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t e = blockIdx.x;
    T* A = lu + e * (size_t)N * LDA;
    auto rowp = [&](int r) -> T* { return A + (size_t)r * LDA; };
    extern __shared__ unsigned char smraw[];
    T* pan = reinterpret_cast<T*>(smraw);   // [N][NB], row index relative to k0
    T* ust = pan + N * NB;                  // [NB][64]
    __shared__ int piv[NB];
    __shared__ T rv[NTH / 32];
    __shared__ int ri[NTH / 32];
    __shared__ int sflag;
    if (tid == 0) sflag = 0;

    // S_r = R_r S R_r^T: block (f, g) of the patch is BSR block blk[e][f][g] (column-major)
#pragma unroll 1
    for (int fg = 0; fg < NF * NF; ++fg) {
        const int f = fg / NF, g = fg - f * NF;
        const T* v = vals + (size_t)blk[e * NF * NF + fg] * BS * BS;
        for (int idx = tid; idx < BS * BS; idx += NTH) {
            const int c = idx / BS, r = idx - c * BS;
            A[(size_t)(f * BS + r) * LDA + g * BS + c] = v[idx];
        }
    }
    __syncthreads();

#pragma unroll 1
    for (int k0 = 0; k0 < N; k0 += NB) {
        const int kb = min(NB, N - k0), nrows = N - k0;
#pragma unroll 1
        for (int idx = tid; idx < nrows * kb; idx += NTH) {
            const int rr = idx / kb, c = idx - rr * kb;
            pan[rr * NB + c] = rowp(k0 + rr)[k0 + c];
        }
        __syncthreads();
#pragma unroll 1
        for (int j = 0; j < kb; ++j) {
            T bv = T(-1);                      // pivot search in the storage type (no FP64 work for FP32)
            int bi = INT_MAX;
#pragma unroll 1
            for (int rr = j + tid; rr < nrows; rr += NTH) {
                const T v = fabs(pan[rr * NB + j]);
                if (v > bv) { bv = v; bi = rr; }
            }
            for (int off = 16; off > 0; off >>= 1) {
                const T ov = __shfl_down_sync(0xffffffffu, bv, off);
                const int oi = __shfl_down_sync(0xffffffffu, bi, off);
                if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
            }
            if (lane == 0) { rv[warp] = bv; ri[warp] = bi; }
            __syncthreads();
            if (tid == 0) {
                T b2 = rv[0];
                int i2 = ri[0];
                for (int w = 1; w < NTH / 32; ++w)
                    if (rv[w] > b2 || (rv[w] == b2 && ri[w] < i2)) { b2 = rv[w]; i2 = ri[w]; }
                if (i2 == INT_MAX) { i2 = j; sflag |= 2; }
                piv[j] = i2;
            }
            __syncthreads();
            const int pr = piv[j];
            if (pr != j)
                for (int c = tid; c < kb; c += NTH) {
                    const T t = pan[j * NB + c];
                    pan[j * NB + c] = pan[pr * NB + c];
                    pan[pr * NB + c] = t;
                }
            __syncthreads();
            T pv = pan[j * NB + j];
            if (pv == T(0) || !isfinite(pv)) {
                if (tid == 0) sflag |= (pv == T(0)) ? 1 : 2;
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
        // interchanges on the columns outside the panel; U12 = L11^{-1} A12 on the right
        const int c0 = k0 + kb;
#pragma unroll 1
        for (int c = tid; c < N; c += NTH) {
            if (c >= k0 && c < c0) continue;
            for (int j = 0; j < kb; ++j) {
                const int pr = piv[j];
                if (pr != j) {
                    T* x = rowp(k0 + j) + c;
                    T* y = rowp(k0 + pr) + c;
                    const T t = *x; *x = *y; *y = t;
                }
            }
            if (c >= c0) {
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
        }
        if (tid < kb) piv_out[e * N + k0 + tid] = k0 + piv[tid];
        __syncthreads();
        trailing_region<T, NB, NTH>(rowp, [&](int j) { return rowp(k0 + j); }, c0, N, c0, N, pan, k0, kb, ust);
    }
    if (tid == 0 && sflag) atomicOr(status, sflag);
}

template <class C>
struct AsmBlk {
    static constexpr int NBLK = (AsmShape<C>::N + 31) / 32;   // 32-row diagonal blocks of the factors
};

// After the factorisation: the row permutation as a gather map (perm[i] = the
// patch row that ends up in row i) and the inverses of the 32 x 32 diagonal
// blocks of L (unit) and U, stored transposed (inv[c][i]) so that a solve
// reads them coalesced.  A partial last block is padded with the identity.
template <class C, class T, int NTH>
__global__ void __launch_bounds__(NTH) k_asm_prep(const T* __restrict__ lu, const int32_t* __restrict__ piv,
                                                  int32_t* __restrict__ perm, T* __restrict__ dinv) {
    constexpr int N = AsmShape<C>::N, LDA = AsmShape<C>::LDA, NBLK = AsmBlk<C>::NBLK;
    __shared__ int p[N];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t e = blockIdx.x;
    const T* A = lu + e * (size_t)N * LDA;
    for (int i = tid; i < N; i += NTH) p[i] = i;
    __syncthreads();
    if (tid == 0)
        for (int i = 0; i < N; ++i) {
            const int q = piv[e * N + i];
            if (q != i) { const int t = p[i]; p[i] = p[q]; p[q] = t; }
        }
    __syncthreads();
    for (int i = tid; i < N; i += NTH) perm[e * N + i] = p[i];
    // lane c of a warp computes column c of inv(L_kk) and of inv(U_kk)
    for (int kb = warp; kb < NBLK; kb += NTH / 32) {
        const int k0 = 32 * kb, nb = min(32, N - k0);
        T* DL = dinv + ((size_t)e * NBLK + kb) * 2048;
        T* DU = DL + 1024;
        double x[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {             // L x = e_c, L unit lower
            double s = (i == lane) ? 1.0 : 0.0;
            if (i < nb) {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j < i) s -= (double)A[(size_t)(k0 + i) * LDA + k0 + j] * x[j];
            }
            x[i] = s;
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) DL[lane * 32 + i] = (T)x[i];
#pragma unroll
        for (int i = 31; i >= 0; --i) {            // U x = e_c
            double s = (i == lane) ? 1.0 : 0.0;
            if (i < nb) {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j > i && j < nb) s -= (double)A[(size_t)(k0 + i) * LDA + k0 + j] * x[j];
                s /= (double)A[(size_t)(k0 + i) * LDA + k0 + i];
            }
            x[i] = s;
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) DU[lane * 32 + i] = (T)x[i];
    }
}

// z_r = S_r^{-1} R_r x for every element r: permuted gather, then blocked
// forward and backward substitution (diagonal blocks by their stored
// inverses, off-diagonal blocks as one dot product per row and thread).  The
// arithmetic runs in the storage type T: FP64 for the FP64 system; FP32 for
// the mixed one, where FP64 work would bound the kernel (GB300 has 1/64 of
// the FP32 rate in FP64) and the FP32 factors fix the accuracy anyway.
template <class T, int NB>
__device__ __forceinline__ T row_dot(const T* __restrict__ a, const T* __restrict__ x, int nb) {
    T s = T(0);
    if (nb == 32) {
        if (sizeof(T) == 4) {
            const float4* a4 = reinterpret_cast<const float4*>(a);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float4 v = __ldg(a4 + j);
                s = fma((T)v.x, x[4 * j], s);
                s = fma((T)v.y, x[4 * j + 1], s);
                s = fma((T)v.z, x[4 * j + 2], s);
                s = fma((T)v.w, x[4 * j + 3], s);
            }
        } else {
            const double2* a2 = reinterpret_cast<const double2*>(a);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const double2 v = __ldg(a2 + j);
                s = fma((T)v.x, x[2 * j], s);
                s = fma((T)v.y, x[2 * j + 1], s);
            }
        }
    } else {
        for (int j = 0; j < nb; ++j) s = fma(a[j], x[j], s);
    }
    return s;
}

template <class C, class T, int NTH>
__global__ void __launch_bounds__(NTH) k_asm_solve(const T* __restrict__ lu, const int32_t* __restrict__ perm,
                                                   const T* __restrict__ dinv, const int32_t* __restrict__ e2f,
                                                   const double* __restrict__ x, double* __restrict__ z) {
    constexpr int N = AsmShape<C>::N, LDA = AsmShape<C>::LDA, NF = C::NF, BS = C::BS;
    constexpr int NBLK = AsmBlk<C>::NBLK, NW = NTH / 32;
    static_assert(NTH == 256, "diagonal-block product assumes 8 warps");
    __shared__ __align__(16) T xs[N];
    __shared__ T red[NW][32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t e = blockIdx.x;
    const T* A = lu + e * (size_t)N * LDA;
    for (int i = tid; i < N; i += NTH) {
        const int j = perm[e * N + i], f = j / BS;
        xs[i] = (T)x[(size_t)e2f[e * NF + f] * BS + (j - f * BS)];
    }
    __syncthreads();
    // xs[k0 .. k0+32) <- inv(D_kk) xs[k0 .. k0+32): warp w sums columns 4w .. 4w+3
    auto diag_product = [&](const T* Dt, int k0, int nb) {
        T s = T(0);
        if (lane < nb) {
#pragma unroll
            for (int c = 4 * warp; c < 4 * warp + 4; ++c)
                if (c < nb) s = fma(Dt[c * 32 + lane], xs[k0 + c], s);
        }
        red[warp][lane] = s;
        __syncthreads();
        if (tid < nb) {
            T t = T(0);
#pragma unroll
            for (int w = 0; w < NW; ++w) t += red[w][tid];
            xs[k0 + tid] = t;
        }
        __syncthreads();
    };
    // xs[r] -= A[r][k0 .. k0+nb) . xs[k0 .. k0+nb) for r in [r0, r1)
    auto offdiag_update = [&](int k0, int nb, int r0, int r1) {
#pragma unroll 1
        for (int r = r0 + tid; r < r1; r += NTH) xs[r] -= row_dot<T, 32>(A + (size_t)r * LDA + k0, xs + k0, nb);
        __syncthreads();
    };
    const T* D = dinv + (size_t)e * NBLK * 2048;
#pragma unroll 1
    for (int kb = 0; kb < NBLK; ++kb) {
        const int k0 = 32 * kb, nb = min(32, N - k0);
        diag_product(D + (size_t)kb * 2048, k0, nb);
        if (k0 + nb < N) offdiag_update(k0, nb, k0 + nb, N);
    }
#pragma unroll 1
    for (int kb = NBLK - 1; kb >= 0; --kb) {
        const int k0 = 32 * kb, nb = min(32, N - k0);
        diag_product(D + (size_t)kb * 2048 + 1024, k0, nb);
        if (k0 > 0) offdiag_update(k0, nb, 0, k0);
    }
    for (int i = tid; i < N; i += NTH) z[e * (size_t)N + i] = (double)xs[i];
}

// y_F = sum over the (one or two) elements of face F of their patch corrections, side 0 first
template <class C>
__global__ void k_asm_sum(const double* __restrict__ z, const int32_t* __restrict__ f2e,
                          const int32_t* __restrict__ f2lf, double* __restrict__ y, int64_t F) {
    constexpr int BS = C::BS, N = AsmShape<C>::N;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= F * BS) return;
    const int64_t f = i / BS;
    const int r = (int)(i - f * BS);
    const int e0 = f2e[2 * f], e1 = f2e[2 * f + 1];
    double s = z[(size_t)e0 * N + f2lf[2 * f] * BS + r];
    if (e1 >= 0) s += z[(size_t)e1 * N + f2lf[2 * f + 1] * BS + r];
    y[i] = s;
}

template <int D, int P>
int run_asm_setup(hdg_ctx* h) {
    using C = Cfg<D, P>;
    constexpr int N = AsmShape<C>::N;
    if (h->sys_prec == HDG_PREC_MIXED) {
        constexpr int NB = 16;
        const int smem = asm_factor_smem_bytes<float, NB>(N);
        HDG_CK(cudaFuncSetAttribute(k_asm_factor<C, float, NB, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        k_asm_factor<C, float, NB, 256><<<(unsigned)h->E, 256, smem, h->stream>>>(
            h->d_vals32, h->d_blk, (float*)h->d_asmlu, h->d_asmpiv, h->d_status);
    } else {
        constexpr int NB = 8;
        const int smem = asm_factor_smem_bytes<double, NB>(N);
        HDG_CK(cudaFuncSetAttribute(k_asm_factor<C, double, NB, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        k_asm_factor<C, double, NB, 256><<<(unsigned)h->E, 256, smem, h->stream>>>(
            h->d_vals, h->d_blk, (double*)h->d_asmlu, h->d_asmpiv, h->d_status);
    }
    if (h->sys_prec == HDG_PREC_MIXED)
        k_asm_prep<C, float, 256><<<(unsigned)h->E, 256, 0, h->stream>>>((const float*)h->d_asmlu, h->d_asmpiv,
                                                                        h->d_asmperm, (float*)h->d_asmdinv);
    else
        k_asm_prep<C, double, 256><<<(unsigned)h->E, 256, 0, h->stream>>>((const double*)h->d_asmlu, h->d_asmpiv,
                                                                         h->d_asmperm, (double*)h->d_asmdinv);
    HDG_CK(cudaGetLastError());
    return HDG_OK;
}

template <int D, int P>
int run_asm_apply(hdg_ctx* h, const double* x, double* y) {
    using C = Cfg<D, P>;
    if (h->asm_prec == HDG_PREC_MIXED)
        k_asm_solve<C, float, 256><<<(unsigned)h->E, 256, 0, h->stream>>>(
            (const float*)h->d_asmlu, h->d_asmperm, (const float*)h->d_asmdinv, h->d_e2f, x, h->d_asmz);
    else
        k_asm_solve<C, double, 256><<<(unsigned)h->E, 256, 0, h->stream>>>(
            (const double*)h->d_asmlu, h->d_asmperm, (const double*)h->d_asmdinv, h->d_e2f, x, h->d_asmz);
    const int64_t n = h->F * C::BS;
    k_asm_sum<C><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->d_asmz, h->d_f2e, h->d_f2lf, y, h->F);
    HDG_CK(cudaGetLastError());
    return HDG_OK;
}

}  // namespace hdg
