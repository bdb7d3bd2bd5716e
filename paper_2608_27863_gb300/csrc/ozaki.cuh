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
// k_oz_scales first computes every row's and column's exponent once per element.
// Then one CTA (16 warps) per (element, 128-row tile, 64-column tile) walks K in
// 32-wide chunks: the raw FP64 tiles of the next chunk are loaded into shared
// memory by TMA (cp.async.bulk.tensor, completing on an mbarrier) while the
// tensor cores run the current one; the threads cut
// the current raw tiles into the s digit slices of its W rows and Z columns, in
// the canonical K-major layout without swizzle (8-row x 16-byte core matrices,
// K-adjacent cores 128 B apart, 8-row groups 512 B apart), and one thread
// issues tcgen05.mma kind::f16 (BF16 inputs, FP32 accumulation in tensor
// memory) for every kept digit pair.  The epilogue combines the six
// accumulators exactly as 64-bit integers and converts once to FP64.  Waits on the MMA completion barrier are
// bounded; on timeout the CTA latches status bit 4, waits once more (bounded)
// and frees its tensor memory.
#pragma once

#include <climits>
#include <cstdint>

#include <cuda.h>

#include "common.h"
#include "tc_util.cuh"

namespace hdg {

constexpr int OZ_THREADS = 512;

template <class C>
struct OzakiCfg {
    static constexpr int K = C::NU, NT = C::NT;
    // digit width: 5 K (2^b - 1)^2 < 2^24 keeps the groups k <= 6 exact
    static constexpr int B = (5LL * K * 255 * 255 < (1LL << 24)) ? 8 : (5LL * K * 127 * 127 < (1LL << 24)) ? 7 : 6;
    static constexpr int S = (54 + B - 1) / B;            // digits: b s >= 54
    static constexpr int NACC = 6;                        // groups 2 .. 6 and the rest
    static constexpr int MT = 128, NTN = 64, KC = 32;
    static constexpr int NMT = (NT + MT - 1) / MT, NNT = (NT + NTN - 1) / NTN;
    static constexpr int TCOLS = 512;                     // NACC * NTN = 384 columns allocated as 512
    static constexpr int A_SLICE = MT * KC * 2, B_SLICE = NTN * KC * 2;   // bytes of one digit slice
    static constexpr int WRS = KC + 2;                    // raw W tile row (doubles): the TMA box is 2 wider than
                                                          // the chunk, which also makes the rows conflict-free
    static constexpr int ZRS = NTN + 2;                   // raw Z tile row: the box starts at an even column
    static constexpr int RAW = (MT * WRS + KC * ZRS) * 8; // raw FP64 tiles of the next chunk
    static constexpr int LOAD_BYTES = RAW;                // bytes one chunk's two TMA loads deliver
    static constexpr int SMEM = S * (A_SLICE + B_SLICE) + RAW + (MT + NTN) * 4 + 64 + 16;
    static_assert((S * (A_SLICE + B_SLICE)) % 128 == 0 && (MT * WRS * 8) % 128 == 0, "TMA destinations 128-B aligned");
    static_assert(S <= 9 && B * S >= 54 && B * S <= 56, "digit layout");
    static_assert(NACC * NTN <= TCOLS, "tensor-memory columns");
    static_assert((5LL * K * ((1 << B) - 1) * ((1 << B) - 1)) < (1LL << 24), "exact FP32 group accumulation");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// exponent e with |v| < 2^e for a normal FP64 value with bits u; zero / subnormal -> INT_MIN
__device__ __forceinline__ int oz_exponent(unsigned long long u) {
    const int E = (int)((u >> 52) & 0x7FF);
    return E == 0 ? INT_MIN : E - 1022;
}

// trunc(|v| 2^{BS - e}) as an integer (< 2^BS <= 2^56) from the FP64 bits u of v
// (|v| < 2^e); zero or subnormal -> 0
__device__ __forceinline__ unsigned long long oz_fixed(unsigned long long u, int e, int BS) {
    const int E = (int)((u >> 52) & 0x7FF);
    const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = e - BS + 1075 - E;                       // |v| 2^{BS - e} = m 2^{-sh}, sh >= 53 - BS
    if (E == 0 || sh >= 64) return 0ull;
    return sh >= 0 ? (m >> sh) : (m << (-sh));
}

// BF16 bits of the signed integer d (|d| < 256) times scale (a power of two): the float
// of d by the magic-number addition 1.5 2^23 + d (exact for |d| < 2^22), scaled, then
// its upper half, which is exact because d has at most 8 significant bits
__device__ __forceinline__ uint32_t oz_digit_bf16(int d, float scale) {
    return __float_as_uint((__int_as_float(0x4B400000 + d) - 12582912.0f) * scale) >> 16;
}

// 2^p as a float (compile-time p in the normal range)
__host__ __device__ constexpr float oz_pow2(int p) {
    return p >= 0 ? float(1ull << (p > 62 ? 62 : p)) : 1.0f / float(1ull << (-p > 62 ? 62 : -p));
}

// the S digit slices (8 K-adjacent values of one row / column) of the values with FP64
// bits u[0..7], scale exponent e, stored as S 16-byte core-matrix rows at dst + i * stride
template <int S, int B, int SHIFT0>
__device__ __forceinline__ void oz_store_digits(const unsigned long long (&u)[8], int e, unsigned char* dst,
                                                int stride) {
    constexpr int BS = B * S;
    unsigned long long F[8];
    int sm[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        F[v] = oz_fixed(u[v], e, BS);
        sm[v] = -(int)(u[v] >> 63);                         // 0 or -1: the sign of the value
    }
#pragma unroll
    for (int i = 0; i < S; ++i) {
        constexpr int mask = (1 << B) - 1;
        const float scale = oz_pow2(-B * (i + 1 - SHIFT0));  // slice i (digit i + 1) staged times 2^{-b (i + 1 - SHIFT0)}
        uint32_t w[4];
#pragma unroll
        for (int v = 0; v < 8; v += 2) {
            int d0 = (int)((F[v] >> (B * (S - 1 - i))) & mask);
            int d1 = (int)((F[v + 1] >> (B * (S - 1 - i))) & mask);
            d0 = (d0 ^ sm[v]) - sm[v];
            d1 = (d1 ^ sm[v + 1]) - sm[v + 1];
            w[v >> 1] = oz_digit_bf16(d0, scale) | (oz_digit_bf16(d1, scale) << 16);
        }
        *reinterpret_cast<uint4*>(dst + i * stride) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// exact accumulator value (FP32 bits: an integer times a power of two) times 2^c as a
// 64-bit integer (the shared "rest" accumulator rounds toward zero below 2^-c)
__device__ __forceinline__ long long oz_acc_fixed(uint32_t bits, int c) {
    const int ea = (int)((bits >> 23) & 0xFF);
    if (ea == 0) return 0ll;
    const long long m = (long long)((bits & 0x7FFFFFu) | 0x800000u);
    const int sh = ea - 150 + c;                               // value 2^c = m 2^{sh}
    const long long v = sh >= 0 ? (m << sh) : (sh <= -64 ? 0ll : (m >> (-sh)));
    return (bits >> 31) ? -v : v;
}

// Scale exponents of one element, written to ex[el][0..NT) (rows of W, one warp per
// row with lanes along the row) and ex[el][NT..2NT) (columns of Z, one thread per
// column, coalesced over the columns): e with every |value| < 2^e, 0 for zero rows.
template <class C>
__global__ void __launch_bounds__(256) k_oz_scales(const double* top, const double* bot, int64_t e0, int32_t* ex) {
    constexpr int NU = C::NU, NT = C::NT, LD = C::LD;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t el = blockIdx.x, e = e0 + el;
    const unsigned long long* Wb = reinterpret_cast<const unsigned long long*>(bot + el * (size_t)NT * LD);
    const unsigned long long* Zb = reinterpret_cast<const unsigned long long*>(top + e * (size_t)NU * LD + NU);
    int32_t* out = ex + el * 2 * NT;
    for (int r = warp; r < NT; r += 8) {
        int m = INT_MIN;
#pragma unroll 4
        for (int k = lane; k < NU; k += 32) m = max(m, oz_exponent(Wb[(size_t)r * LD + k]));
        m = __reduce_max_sync(0xffffffffu, m);
        if (lane == 0) out[r] = m == INT_MIN ? 0 : m;
    }
    for (int c = tid; c < NT; c += 256) {
        int m = INT_MIN;
#pragma unroll 8
        for (int k = 0; k < NU; ++k) m = max(m, oz_exponent(Zb[(size_t)k * LD + c]));
        out[NT + c] = m == INT_MIN ? 0 : m;
    }
}

// W tiles: tmW over the chunk's trace rows [chunk][NT][LD] (box 34 x 128); Z tiles: tmZ
// over the interior rows [E][NU][LD] (box 66 x 32, starting at the even column at or
// below NU + n0); rows past NT (W) or NU (Z) and columns past LD arrive as zeros.
template <class C>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_schur_ozaki(double* top, double* bot, int64_t e0, const int32_t* ex,
                                                               int32_t* status, const __grid_constant__ CUtensorMap tmW,
                                                               const __grid_constant__ CUtensorMap tmZ) {
    using O = OzakiCfg<C>;
    constexpr int NU = C::NU, NT = C::NT, LD = C::LD;
    constexpr int MT = O::MT, NTN = O::NTN, KC = O::KC, S = O::S, B = O::B, WRS = O::WRS, ZRS = O::ZRS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t bid = blockIdx.x;
    const int nt = (int)(bid % O::NNT), mt = (int)((bid / O::NNT) % O::NMT);
    const int64_t el = bid / (O::NNT * O::NMT), e = e0 + el;
    const int m0 = mt * MT, n0 = nt * NTN;
    double* Bm = bot + el * (size_t)NT * LD;                    // S_rc at Bm[r * LD + NU + c]
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* As = smraw;                                  // S slices [MT rows][KC] BF16, core layout
    unsigned char* Bs = As + S * O::A_SLICE;                    // S slices [NTN cols][KC]
    unsigned long long* Wr = reinterpret_cast<unsigned long long*>(Bs + S * O::B_SLICE);   // [MT][WRS] raw W
    unsigned long long* Zr = Wr + MT * WRS;                     // [KC][ZRS] raw Z
    int* er = reinterpret_cast<int*>(Zr + KC * ZRS);            // [MT] row exponents
    int* fc = er + MT;                                          // [NTN] column exponents
    uint64_t* mbar = reinterpret_cast<uint64_t*>(fc + NTN);    // [0] MMA completion, [1] TMA loads
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);

    // raw FP64 tiles of the chunk starting at k0, loaded by the tensor memory accelerator
    const int zx = (NU + n0) & ~1, zoff = (NU + n0) & 1;        // Z box column start (even) and the offset in it
    const uint32_t bar_ld = smem_u32(mbar + 1);
    uint32_t ld_phase = 0;
    bool ld_pending = false;                                    // a load is in flight (all threads track it)
    auto prefetch = [&](int k0) {
        ld_pending = true;
        if (tid == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar_ld), "r"(O::LOAD_BYTES)
                         : "memory");
            asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                         "[%0], [%1, {%2, %3, %4}], [%5];"
                         :: "r"(smem_u32(Wr)), "l"(reinterpret_cast<uint64_t>(&tmW)), "r"(k0), "r"(m0), "r"((int)el),
                            "r"(bar_ld) : "memory");
            asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                         "[%0], [%1, {%2, %3, %4}], [%5];"
                         :: "r"(smem_u32(Zr)), "l"(reinterpret_cast<uint64_t>(&tmZ)), "r"(zx), "r"(k0), "r"((int)e),
                            "r"(bar_ld) : "memory");
        }
    };
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar_ld), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    prefetch(0);

    // row and column scales of this tile (k_oz_scales)
    for (int i = tid; i < MT; i += OZ_THREADS) er[i] = m0 + i < NT ? ex[el * 2 * NT + m0 + i] : 0;
    for (int i = tid; i < NTN; i += OZ_THREADS) fc[i] = n0 + i < NT ? ex[el * 2 * NT + NT + n0 + i] : 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(tslot)),
                     "r"(O::TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
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
    bool ok = true, pending = false;                            // an MMA batch reads the digit slices
    unsigned used = 0;                                          // accumulators written so far (thread 0)
    for (int k0 = 0; k0 < NU; k0 += KC) {
        if (!mbar_wait_bounded(bar_ld, ld_phase, 1 << 24)) {   // this chunk's tiles have landed
            ok = false;
            if (tid == 0) atomicOr(status, 4);
            mbar_wait_bounded(bar_ld, ld_phase, 1 << 24);
        }
        ld_phase ^= 1;
        ld_pending = false;
        if (pending) {                                          // the previous batch still reads the slices
            if (!mbar_wait_bounded(bar, phase, 1 << 24)) {
                ok = false;
                if (tid == 0) atomicOr(status, 4);
                mbar_wait_bounded(bar, phase, 1 << 24);
            }
            phase ^= 1;
            pending = false;
        }
        // raw tiles of this chunk visible, slices free; a timed-out wait stops every thread
        if (__syncthreads_or(ok ? 0 : 1)) {
            ok = false;
            break;
        }
        // A: item = (row r, 8-wide K group q), rows fastest
        for (int it = tid; it < MT * (KC / 8); it += OZ_THREADS) {
            const int r = it % MT, q = it / MT;
            unsigned long long u[8];
            const ulonglong2* src = reinterpret_cast<const ulonglong2*>(Wr + r * WRS + q * 8);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const ulonglong2 x = src[v];
                u[2 * v] = x.x;
                u[2 * v + 1] = x.y;
            }
#pragma unroll
            for (int v = 0; v < 8; ++v) if (k0 + q * 8 + v >= NU) u[v] = 0ull;   // trace columns: not W
            const int off = ((r >> 3) * (KC / 8) + q) * 128 + (r & 7) * 16;
            oz_store_digits<S, B, 3>(u, er[r], As + off, O::A_SLICE);
        }
        // B: item = (column n, 8-wide K group q), columns fastest
        for (int it = tid; it < NTN * (KC / 8); it += OZ_THREADS) {
            const int n = it % NTN, q = it / NTN;
            unsigned long long u[8];
#pragma unroll
            for (int v = 0; v < 8; ++v) u[v] = n0 + n < NT ? Zr[(q * 8 + v) * ZRS + zoff + n] : 0ull;
            const int off = ((n >> 3) * (KC / 8) + q) * 128 + (n & 7) * 16;
            oz_store_digits<S, B, 4>(u, fc[n], Bs + off, O::B_SLICE);
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();                                        // slices written, raw tiles consumed
        if (k0 + KC < NU) prefetch(k0 + KC);                    // next chunk's tiles under this chunk's MMAs
        // (the fence.proxy.async above orders this CTA's reads of the raw tiles before the loads)
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
        pending = true;
    }
    if (ld_pending) mbar_wait_bounded(bar_ld, ld_phase, 1 << 24);   // after an early stop: no copy outlives the CTA
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
        // warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (tile rows) and the 16-column
        // quarter w / 4 of the tile; the six accumulators are combined exactly as integers in
        // units of 2^{5b - 38} (the leading group needs at most 62 bits), converted once to FP64,
        // scaled by 2^{e_r + f_c - 2b - 38} and subtracted from Dt
        const int lg = warp & 3, c0 = (warp >> 2) * 16;
        const int r = lg * 32 + lane, row = m0 + r;
        long long tot[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) tot[j] = 0ll;
#pragma unroll 1
        for (int g = 0; g < O::NACC; ++g) {
            uint32_t v[16];
            const uint32_t addr = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(g * NTN + c0);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                           "=r"(v[14]), "=r"(v[15])
                         : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            // accumulator g holds a group only if some kept digit pair falls in it
            if (g < 5 ? (g + 2 <= S + 1) : (S + 1 >= 7)) {
#pragma unroll
                for (int j = 0; j < 16; ++j) tot[j] += oz_acc_fixed(v[j], 38 - 5 * B);
            }
        }
        if (row < NT) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int c = n0 + c0 + j;
                if (c < NT) {
                    const int sc = er[r] + fc[c0 + j] - 2 * B - 38;
                    const double x = __ll2double_rn(tot[j]);
                    double* sp = Bm + (size_t)row * LD + NU + c;
                    if (sc > -1023 && sc < 1024)               // 2^sc as a normal double, from its bits
                        *sp -= x * __longlong_as_double((long long)(1023 + sc) << 52);
                    else
                        *sp -= ldexp(x, sc);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(O::TCOLS));
}

}  // namespace hdg
