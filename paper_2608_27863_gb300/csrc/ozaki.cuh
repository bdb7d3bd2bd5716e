// FP64 Schur product S^K = Dt - W Z emulated on the 5th-generation tensor
// cores (the error-free splitting of Ozaki, Ogita, Oishi and Rump, 2012), for
// the FP64 form: W = Ct U^{-1} (trace rows x interior columns, the multipliers
// the bordered elimination leaves in the trace rows) and Z = L^{-1} P Bt
// (interior rows x trace columns) stay in FP64 in HBM; only their products
// run on the BF16 tensor pipe.
//
// Splitting.  Row r of W is scaled by 2^{-e_r} (e_r the smallest power of two
// above max_k |W_rk|) and column c of Z by 2^{-f_c}; each scaled value is cut,
// by integer operations on its FP64 bits, into s digits of b bits:
//     W_rk ~ 2^{e_r} sum_i 2^{-b i} a_i,   Z_kc ~ 2^{f_c} sum_j 2^{-b j} z_j,
// with integer digits |a_i|, |z_j| < 2^b carrying the value's sign (truncation
// error below 2^{-b s} of the row / column scale; b s >= 54).  A digit times
// a power of two is exact in BF16 (8 significant bits, b <= 8).  The integer
// products A_i Z_j (K = n_u terms) are exact in the FP32 accumulator as long
// as every partial sum stays below 2^24: with b chosen so that
// 5 n_u (2^b - 1)^2 < 2^24, the pairs of each digit-sum group k = i + j <= 6
// accumulate exactly into their own accumulator.  Pairs with k >= 7, whose
// weight is 2^{-5b} or less relative to the leading group, share one
// accumulator; pairs with k > s + 1 are dropped (below the truncation error).
// Slices are staged pre-scaled by 2^{-b (i - 3)} and 2^{-b (j - 4)}, so every
// accumulator holds 2^{-b (k - 7)} G_k (G_k = sum over i + j = k of A_i Z_j)
// and the six accumulators sum to 2^{7b} 2^{-e_r - f_c} (W Z)_rc; the epilogue
// adds them in FP64, scales and subtracts from Dt in FP64.
//
// One CTA (4 warps) per (element, 128-row tile, 32-column tile): the CTA
// computes its rows' and columns' exponents, then for each 32-wide K chunk
// stages the s digit slices of its W rows and Z columns in shared memory in
// the canonical K-major layout without swizzle (8-row x 16-byte core matrices,
// K-adjacent cores 128 B apart, 8-row groups 512 B apart) and one thread
// issues tcgen05.mma kind::f16 (BF16 inputs, FP32 accumulation in tensor
// memory) for every kept digit pair.  Waits on the MMA completion barrier are
// bounded; on timeout the CTA latches status bit 4, waits once more (bounded)
// and frees its tensor memory.
#pragma once

#include <cuda_bf16.h>

#include "mixed.cuh"

namespace hdg {

template <class C>
struct OzakiCfg {
    static constexpr int K = C::NU, NT = C::NT;
    // digit width: 5 K (2^b - 1)^2 < 2^24 keeps the groups k <= 6 exact
    static constexpr int B = (5LL * K * 255 * 255 < (1LL << 24)) ? 8 : (5LL * K * 127 * 127 < (1LL << 24)) ? 7 : 6;
    static constexpr int S = (54 + B - 1) / B;            // digits: b s >= 54
    static constexpr int NACC = 6;                        // groups 2 .. 6 and the rest
    static constexpr int MT = 128, NTN = 32, KC = 32;
    static constexpr int NMT = (NT + MT - 1) / MT, NNT = (NT + NTN - 1) / NTN;
    static constexpr int TCOLS = 256;                     // NACC * NTN = 192 columns allocated as 256
    static constexpr int A_SLICE = MT * KC * 2, B_SLICE = NTN * KC * 2;   // bytes of one digit slice
    static constexpr int SMEM = S * (A_SLICE + B_SLICE) + (MT + NTN) * 4 + 64;
    static_assert(S <= 9 && B * S >= 54, "digit layout");
    static_assert(NACC * NTN <= TCOLS, "tensor-memory columns");
    static_assert((5LL * K * ((1 << B) - 1) * ((1 << B) - 1)) < (1LL << 24), "exact FP32 group accumulation");
};

// exponent e with |v| < 2^e for a normal FP64 v, from its bits; zero / subnormal -> INT_MIN
__device__ __forceinline__ int oz_exponent(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const int E = (int)((u >> 52) & 0x7FF);
    return E == 0 ? INT_MIN : E - 1022;
}

// trunc(|v| 2^{BS - e}) as an integer (< 2^BS), from the FP64 bits; v == 0 or subnormal -> 0
__device__ __forceinline__ unsigned long long oz_fixed(double v, int e, int BS) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const int E = (int)((u >> 52) & 0x7FF);
    if (E == 0) return 0ull;
    const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = (E - 1075) + BS - e;                     // |v| 2^{BS - e} = m 2^{sh}
    if (sh >= 0) return m << sh;                            // sh <= BS - 53 + ... < 64 since |v| < 2^e
    return sh <= -64 ? 0ull : (m >> (-sh));
}

// BF16 bits of the integer d (|d| < 256) times 2^{p}: exact
__device__ __forceinline__ uint16_t oz_bf16(int d, int p) {
    if (d == 0) return 0;
    const uint32_t s = d < 0 ? 0x8000u : 0u;
    const uint32_t a = (uint32_t)(d < 0 ? -d : d);
    const int msb = 31 - __clz(a);                          // a = 1.f x 2^msb
    const uint32_t frac = (a << (7 - msb)) & 0x7Fu;          // 7 fraction bits (a has <= 8 bits)
    return (uint16_t)(s | ((uint32_t)(127 + msb + p) << 7) | frac);
}

template <class C>
__global__ void __launch_bounds__(128) k_schur_ozaki(double* top, double* bot, int64_t e0, int32_t* status) {
    using O = OzakiCfg<C>;
    constexpr int NU = C::NU, NT = C::NT, LD = C::LD;
    constexpr int MT = O::MT, NTN = O::NTN, KC = O::KC, S = O::S, B = O::B, BS = O::B * O::S;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t bid = blockIdx.x;
    const int nt = (int)(bid % O::NNT), mt = (int)((bid / O::NNT) % O::NMT);
    const int64_t el = bid / (O::NNT * O::NMT), e = e0 + el;
    const int m0 = mt * MT, n0 = nt * NTN;
    const double* Z = top + e * (size_t)NU * LD + NU;          // Z_kc at Z[k * LD + c]
    double* Bm = bot + el * (size_t)NT * LD;                    // W_rk at Bm[r * LD + k], S_rc at Bm[r * LD + NU + c]
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* As = smraw;                                  // S slices [MT rows][KC] BF16, core layout
    unsigned char* Bs = smraw + S * O::A_SLICE;                 // S slices [NTN cols][KC]
    int* er = reinterpret_cast<int*>(Bs + S * O::B_SLICE);      // [MT] row exponents
    int* fc = er + MT;                                          // [NTN] column exponents
    uint64_t* mbar = reinterpret_cast<uint64_t*>(fc + NTN);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);

    // row and column scales
    {
        const int r = m0 + tid;
        int m = INT_MIN;
        if (tid < MT && r < NT)
            for (int k = 0; k < NU; ++k) m = max(m, oz_exponent(Bm[(size_t)r * LD + k]));
        er[tid] = m == INT_MIN ? 0 : m;
    }
    if (tid < NTN) {
        const int c = n0 + tid;
        int m = INT_MIN;
        if (c < NT)
            for (int k = 0; k < NU; ++k) m = max(m, oz_exponent(Z[(size_t)k * LD + c]));
        fc[tid] = m == INT_MIN ? 0 : m;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(tslot)),
                     "r"(O::TCOLS));
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
    // kind::f16: F32 accumulator, BF16 A and B, both K-major, N = NTN, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NTN >> 3) << 17) |
                           ((uint32_t)(MT >> 4) << 24);
    const uint32_t bar = smem_u32(mbar);
    uint32_t phase = 0;
    bool ok = true;
    unsigned used = 0;                                          // accumulators written so far (thread 0)
    for (int k0 = 0; k0 < NU; k0 += KC) {
        // A: item = (row r, 8-wide K group q): 8 FP64 values -> S slices of 8 BF16 (16 bytes each)
        for (int it = tid; it < MT * (KC / 8); it += 128) {
            const int r = it / (KC / 8), q = it - r * (KC / 8);
            const int row = m0 + r;
            uint16_t dig[S][8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + q * 8 + u;
                const double v = (row < NT && k < NU) ? Bm[(size_t)row * LD + k] : 0.0;
                const unsigned long long F = oz_fixed(v, er[r], BS);
                const bool neg = v < 0.0;
#pragma unroll
                for (int i = 0; i < S; ++i) {
                    const int d = (int)((F >> (B * (S - 1 - i))) & ((1u << B) - 1));
                    dig[i][u] = oz_bf16(neg ? -d : d, -B * (i + 1 - 3));      // 2^{-b (i - 3)}, i from 1
                }
            }
            // core matrix (8-row group r / 8, K group q): offset ((r / 8) * (KC / 8) + q) * 128 + (r % 8) * 16
            const int off = ((r >> 3) * (KC / 8) + q) * 128 + (r & 7) * 16;
#pragma unroll
            for (int i = 0; i < S; ++i) {
                uint4 w;
                w.x = dig[i][0] | ((uint32_t)dig[i][1] << 16);
                w.y = dig[i][2] | ((uint32_t)dig[i][3] << 16);
                w.z = dig[i][4] | ((uint32_t)dig[i][5] << 16);
                w.w = dig[i][6] | ((uint32_t)dig[i][7] << 16);
                *reinterpret_cast<uint4*>(As + i * O::A_SLICE + off) = w;
            }
        }
        // B: item = (column n, 8-wide K group q)
        for (int it = tid; it < NTN * (KC / 8); it += 128) {
            const int n = it % NTN, q = it / NTN;
            const int col = n0 + n;
            uint16_t dig[S][8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + q * 8 + u;
                const double v = (col < NT && k < NU) ? Z[(size_t)k * LD + col] : 0.0;
                const unsigned long long F = oz_fixed(v, fc[n], BS);
                const bool neg = v < 0.0;
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    const int d = (int)((F >> (B * (S - 1 - j))) & ((1u << B) - 1));
                    dig[j][u] = oz_bf16(neg ? -d : d, -B * (j + 1 - 4));      // 2^{-b (j - 4)}
                }
            }
            const int off = ((n >> 3) * (KC / 8) + q) * 128 + (n & 7) * 16;
#pragma unroll
            for (int j = 0; j < S; ++j) {
                uint4 w;
                w.x = dig[j][0] | ((uint32_t)dig[j][1] << 16);
                w.y = dig[j][2] | ((uint32_t)dig[j][3] << 16);
                w.z = dig[j][4] | ((uint32_t)dig[j][5] << 16);
                w.w = dig[j][6] | ((uint32_t)dig[j][7] << 16);
                *reinterpret_cast<uint4*>(Bs + j * O::B_SLICE + off) = w;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int nsteps = (min(KC, NU - k0) + 15) / 16;
            for (int i = 0; i < S; ++i)
                for (int j = 0; j < S; ++j) {
                    const int k = i + j + 2;                    // digit-sum group (digits counted from 1)
                    if (k > S + 1) continue;
                    const int g = k <= 6 ? k - 2 : 5;
                    for (int st = 0; st < nsteps; ++st) {
                        const uint32_t off = st * 256;          // 16 K values = two K-adjacent core matrices
                        const uint64_t da = umma_desc(smem_u32(As + i * O::A_SLICE) + off, 128, (KC / 8) * 128);
                        const uint64_t db = umma_desc(smem_u32(Bs + j * O::B_SLICE) + off, 128, (KC / 8) * 128);
                        const uint32_t acc = (used >> g) & 1u;
                        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                                     :: "r"(tmem + (uint32_t)(g * NTN)), "l"(da), "l"(db), "r"(idesc), "r"(acc));
                        used |= 1u << g;
                    }
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar));
        }
        if (!mbar_wait_bounded(bar, phase, 1 << 24)) {
            ok = false;
            if (tid == 0) atomicOr(status, 4);
            mbar_wait_bounded(bar, phase, 1 << 24);
        }
        phase ^= 1;
        __syncthreads();
        if (!ok) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        // row r of the tile is tensor-memory lane r: warp w reads lanes 32 w .. 32 w + 31
        const int r = warp * 32 + lane, row = m0 + r;
        const int escale = er[r] - 7 * B;
#pragma unroll 1
        for (int c0 = 0; c0 < NTN; c0 += 16) {
            double sum[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) sum[j] = 0.0;
#pragma unroll 1
            for (int g = 0; g < O::NACC; ++g) {
                uint32_t v[16];
                const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(g * NTN + c0);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                               "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                               "=r"(v[14]), "=r"(v[15])
                             : "r"(addr));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                // accumulator g holds a group only if some kept digit pair falls in it
                if (g < 5 ? (g + 2 <= S + 1) : (S + 1 >= 7)) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) sum[j] += (double)__uint_as_float(v[j]);
                }
            }
            if (row < NT) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = n0 + c0 + j;
                    if (c0 + j < NTN && c < NT) {
                        double* s = Bm + (size_t)row * LD + NU + c;
                        *s -= ldexp(sum[j], escale + fc[c0 + j]);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(O::TCOLS));
}

}  // namespace hdg
