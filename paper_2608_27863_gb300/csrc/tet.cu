// Tetrahedral elements of mixed degree on quadratic geometry on the device:
// one persistent FP64 launch performs, element after element from a
// cost-ordered work list, the quadrature-point fluxes and Jacobians (A1), the
// exact elimination of the gradient q (per-element mass matrix and lifting
// operators, curved geometry included), the contraction into the bordered
// element matrix (A2) and its elimination into the Schur complement (A3, A4);
// then the block assembly (A5), the trace matvec (A6) and the interior
// recovery (A7) with variable block sizes, the FP64 stage residual and the
// block-Jacobi preconditioner of the trace system (A8).
#include <algorithm>
#include <climits>
#include <cstring>
#include <type_traits>

#include "kernels.cuh"
#include "solve.cuh"
#include "tet.h"
#include "tet_elim.cuh"

namespace hdg {
namespace tet {

static_assert(sizeof(TetElem) % 8 == 0, "descriptor copied as 64-bit words");

constexpr int NPT = NQMAX + 4 * NFQMAX;   // volume + face points
constexpr int NCM = NPMAX + 4 * NFPMAX;   // columns of one component: U nodes + trace nodes
constexpr int KC = 40;                    // contraction: points staged per step
constexpr int SRP = 36;                   // staged row-basis stride (NPMAX rounded up to 4)
constexpr int STP = 96;                   // staged column stride (NCM rounded up to 4)
constexpr int NB = 16;                    // largest elimination panel width (shared-memory sizing)
constexpr int NRMAX = M * NPMAX + 4 * M * NFPMAX;

// per-CTA workspace layout (doubles)
constexpr int64_t W_GV = 0;                              // [NQMAX][10] w|J|, J^{-1}[r][k]
constexpr int64_t W_GF = W_GV + NQMAX * 10;              // [4 NFQMAX][3] w_s |J| J^{-T} nu
constexpr int64_t W_PU = W_GF + 4 * NFQMAX * 3;          // [NPT][m] u
constexpr int64_t W_PQ = W_PU + NPT * M;                 // [NPT][m][3] q
constexpr int64_t W_PL = W_PQ + NPT * M * 3;             // [NPT][m][3] lifted q
constexpr int64_t W_PH = W_PL + NPT * M * 3;             // [4 NFQMAX][m] uhat
constexpr int64_t W_CV = W_PH + 4 * NFQMAX * M;          // [NQMAX][a][r][b][kind 4]
constexpr int64_t W_CF = W_CV + (int64_t)NQMAX * 300;    // [4 NFQMAX][a][b][kind 5]  element rows (dt folded)
constexpr int64_t W_CB = W_CF + 4 * NFQMAX * 125;        // [4 NFQMAX][a][b][kind 5]  trace rows
constexpr int64_t W_RV = W_CB + 4 * NFQMAX * 125;        // [NQMAX][a][r]
constexpr int64_t W_RF = W_RV + NQMAX * 15;              // [4 NFQMAX][a]
constexpr int64_t W_RB = W_RF + 4 * NFQMAX * M;          // [4 NFQMAX][a]
constexpr int64_t W_MM = W_RB + 4 * NFQMAX * M;          // [NPMAX][NPMAX] mass matrix, then its Cholesky factor
constexpr int64_t W_DP = W_MM + NPMAX * NPMAX;           // [NQMAX][3][NPMAX] physical gradients
constexpr int64_t W_VQ = W_DP + NQMAX * 3 * NPMAX;       // [3][NPT][NCM] psi | chi
constexpr int64_t W_GHF = W_VQ + 3LL * NPT * NCM;       // mixed form: FP32 copies of G | H
constexpr int64_t W_END = W_GHF + (3LL * NPMAX * NCM + 1) / 2;

// shared memory layout (doubles)
constexpr int S_U = 0;                                   // [m][Np]
constexpr int S_US = S_U + M * NPMAX;                    // [m][Np] Ustar
constexpr int S_Q = S_US + M * NPMAX;                    // [3][m][Np]
constexpr int S_QL = S_Q + 3 * M * NPMAX;                // [3][m][Np] lifted gradient
constexpr int S_UH = S_QL + 3 * M * NPMAX;               // [t] element trace
constexpr int S_DYN = S_UH + 4 * M * NFPMAX;             // phase scratch
constexpr int S_GEMM = KC * (SRP + STP);
constexpr int S_ELIM = NRMAX * NB + NB * TCW;
constexpr int S_TOTAL = S_DYN + (S_GEMM > S_ELIM ? S_GEMM : S_ELIM);

struct KArgs {
    const TetElem* el; const int32_t* order; int64_t E; int32_t* next;
    const double* tab; const float* tabf; const double* gvol; const double* gface;
    const double* U; const double* Q; const double* UH; const double* Ustar;
    double* mat; double* rec; double* work; int64_t wstride;
    PhysT<double> ph; PhysT<float> phf;                  // phf: Jacobian terms of the mixed form
    double dt, a_ii, tau; const double* ub; double ew;
    int tau_mode;                                         // 0 constant tau, 1 state-dependent (stab_tau)
    int32_t* status;
    double* Rq; double* Ru; double* rk; double* part;     // residual evaluation outputs
};

__device__ __forceinline__ int face_of_point(const TetElem& d, int r) {
    int f = 0;
    while (f < 3 && r >= d.soff[f + 1]) ++f;
    return f;
}

// element basis row at point x (volume points first, then the face points)
template <class T>
__device__ __forceinline__ const T* basis_row_t(const T* tab, const TetElem& d, int x) {
    if (x < d.Nq) return tab + d.vtab + (size_t)x * d.Np;
    const int r = x - d.Nq, f = face_of_point(d, r);
    return tab + d.ftab[f] + (size_t)(r - d.soff[f]) * d.Np;
}
__device__ __forceinline__ const double* basis_row(const KArgs& A, const TetElem& d, int x) {
    return basis_row_t(A.tab, d, x);
}

// physical constants in the evaluation type of the Jacobian terms
template <class S> __device__ __forceinline__ const PhysT<S>& jphys(const KArgs& A);
template <> __device__ __forceinline__ const PhysT<double>& jphys<double>(const KArgs& A) { return A.ph; }
template <> __device__ __forceinline__ const PhysT<float>& jphys<float>(const KArgs& A) { return A.phf; }

// tables in the contraction type: FP64, or their FP32 copy in the mixed form
template <class T> __device__ __forceinline__ const T* jtab(const KArgs& A);
template <> __device__ __forceinline__ const double* jtab<double>(const KArgs& A) { return A.tab; }
template <> __device__ __forceinline__ const float* jtab<float>(const KArgs& A) { return A.tabf; }


// column index in the bordered matrix of column c (of component b) of the contraction
__device__ __forceinline__ int bcol(const TetElem& d, int b, int c) {
    if (c < d.Np) return b * d.Np + c;
    int r = c - d.Np, f = 0;
    while (f < 3 && r >= d.nfp[f]) { r -= d.nfp[f]; ++f; }
    return d.NU + d.toff[f] + b * d.nfp[f] + r;
}

// one out[i][c] += sum_k R[k][i] T[k][c] pass over a staged chunk; 4 x 4 register tiles
template <class T>
__device__ __forceinline__ void gemm_chunk(const T* sR, const T* sT, int kc, int ti, int tc, T acc[4][4]) {
    for (int k = 0; k < kc; ++k) {
        T rv[4], tv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { rv[u] = sR[k * SRP + 4 * ti + u]; tv[u] = sT[k * STP + 4 * tc + u]; }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(rv[u], tv[v], acc[u][v]);
    }
}


// A0: gather the element's nodal state and trace into shared memory
__device__ void gather_element(const KArgs& A, const TetElem& d, double* sm) {
    const int tid = threadIdx.x, NU = d.NU, t = d.t;
    for (int i = tid; i < NU; i += NTH) { sm[S_U + i] = A.U[d.uoff + i]; sm[S_US + i] = A.Ustar[d.uoff + i]; }
    for (int i = tid; i < 3 * NU; i += NTH) sm[S_Q + i] = A.Q[3 * d.uoff + i];
    for (int i = tid; i < t; i += NTH) {
        int f = 0, r = i;
        while (f < 3 && r >= M * d.nfp[f]) { r -= M * d.nfp[f]; ++f; }
        sm[S_UH + i] = A.UH[d.hoff[f] + r];
    }
}

// geometry at the quadrature points: volume records (w |J|, J^{-1}) and face
// records (w_s |J| J^{-T} nu), from the per-point data of curved elements or the
// affine element's constant Jacobian
__device__ void load_geometry(const KArgs& A, const TetElem& d, double* gv, double* gf) {
    const int tid = threadIdx.x;
    const double* wq = A.tab + d.vtab + (size_t)4 * d.Nq * d.Np;
    for (int g = tid; g < d.Nq; g += NTH) {
        double* o = gv + g * 10;
        if (d.curved) {
            for (int k = 0; k < 10; ++k) o[k] = A.gvol[d.goff + (int64_t)g * 10 + k];
        } else {
            o[0] = wq[g] * d.detJ;
            for (int k = 0; k < 9; ++k) o[1 + k] = d.Jinv[k];
        }
    }
    for (int r = tid; r < d.sfq; r += NTH) {
        double* o = gf + r * 3;
        if (d.curved) {
            for (int k = 0; k < 3; ++k) o[k] = A.gface[d.gfoff + (int64_t)r * 3 + k];
        } else {
            const int f = face_of_point(d, r), s = r - d.soff[f];
            const double* nu = A.tab + d.ftab[f] + (size_t)d.nfq[f] * d.Np;
            const double ws = A.tab[d.ttab[f] + (size_t)d.nfq[f] * d.nfp[f] + s];
            for (int k = 0; k < 3; ++k)
                o[k] = ws * d.detJ * (d.Jinv[0 * 3 + k] * nu[0] + d.Jinv[1 * 3 + k] * nu[1] + d.Jinv[2 * 3 + k] * nu[2]);
        }
    }
}

// ---------------------------------------------------------------------------
// Mixed form: the contraction A2 on the tensor cores.
//
// The column operand of a component pair, T_ab[k][c] = sum_j s_j o_ab[k][j]
// B_j[k][c], is linear in the point coefficients o_ab, so the element rows
// C_ab[i][c] = sum_k R[k][i] T_ab[k][c] are also the product
//   C[(ab, i)][c] = sum_{(j, k)} (s_j R[k][i] o_ab[k][j]) B[(j, k)][c]
// whose column operand B is the same for all 25 pairs: the pairs stack along M
// (25 Np rows) and B is formed once per chunk for all of them.  At a volume
// point g the three directions of R (dphi_r[g][i]) fold into the row operand
// too, since B depends on g only: 4 Nq terms (j = basis, psi/chi 1..3), then
// 5 terms per face point (basis, face trace basis, psi/chi 1..3).  The trace
// rows of face f are the same product with R = mu_f and the trace-row
// coefficients over the points of f.  The products are 3xTF32 (hi hi + hi lo +
// lo hi) accumulated in FP32 in tensor memory; 8 warps form the operands of
// chunk c + 1 while the tensor cores run chunk c.
constexpr int TKC = 16;                       // K per staged chunk
constexpr int TMT = 128;                      // rows per tile (tensor-memory lanes)
constexpr int TNP = 96;                       // columns: Nc <= 95, padded to a multiple of 16
constexpr int TSTAGE = 2 * (TMT + TNP) * TKC; // floats per stage: A hi | B hi | A lo | B lo
constexpr int TTCOLS = 128;                   // tensor-memory columns per CTA
static_assert(2 * TSTAGE * (int)sizeof(float) <= (S_GEMM > S_ELIM ? S_GEMM : S_ELIM) * (int)sizeof(double),
              "two operand stages fit the phase scratch");
static_assert((S_DYN * sizeof(double)) % 16 == 0, "operand stages 16-byte aligned");

struct TcState {        // per CTA, kept over the elements of the persistent loop
    uint32_t tmem;      // accumulator (TTCOLS columns)
    uint32_t bar;       // shared address of two mbarriers, one per operand stage
    uint32_t phase;     // bit s: parity of the next phase of barrier s
};

// four consecutive K entries of one operand row, TF32 hi and lo parts, at the
// row's position in the K-major core-matrix layout (8 rows x 16 bytes)
__device__ __forceinline__ void tc_put4(float* hi, float* lo, int row, int kq, const float v[4]) {
    const int off = ((row >> 3) * (TKC / 4) + kq) * 32 + (row & 7) * 4;
    const float4 h = make_float4(tf32_round(v[0]), tf32_round(v[1]), tf32_round(v[2]), tf32_round(v[3]));
    *reinterpret_cast<float4*>(hi + off) = h;
    *reinterpret_cast<float4*>(lo + off) =
        make_float4(tf32_round(v[0] - h.x), tf32_round(v[1] - h.y), tf32_round(v[2] - h.z), tf32_round(v[3] - h.w));
}

// one segment of the stacked product: the element rows (f = -1) or the trace
// rows of face f.  Its K runs over blocks of one j each (volume j = 0..3 over
// the Nq points, then face j = 0..4 over the sum_f Nfq face points; trace rows:
// j = 0..4 over the Nfq points of face f), every block padded to whole chunks
// so that a chunk has one j and consecutive points.
struct TcSeg {
    int f, rows, rdiv;      // rdiv: rows per pair (Np, or Nfp of face f)
    int cv, cf, nch;        // chunks per volume block, per face block; chunks in all
};

struct TcChunk {
    bool vol;
    int j, p0, np;          // the chunk's points p0 .. p0 + 15 below the block's end np (face points:
                            // an index into the sum_f Nfq face points)
};

__device__ __forceinline__ TcChunk tc_chunk(const TetElem& d, const TcSeg& sg, int ci) {
    TcChunk k;
    if (sg.f < 0 && ci < 4 * sg.cv) {
        k.vol = true; k.j = ci / sg.cv; k.p0 = (ci - k.j * sg.cv) * TKC; k.np = d.Nq;
        return k;
    }
    const int c2 = sg.f < 0 ? ci - 4 * sg.cv : ci;
    k.vol = false; k.j = c2 / sg.cf;
    const int base = sg.f < 0 ? 0 : d.soff[sg.f];
    k.p0 = base + (c2 - k.j * sg.cf) * TKC;
    k.np = base + (sg.f < 0 ? d.sfq : d.nfq[sg.f]);
    return k;
}

// the row of the tile this thread forms: (pair, i), fixed over the chunks of a tile
struct TcRow {
    bool live;
    int i, cvo, cfo;        // basis index; coefficient offsets of the pair in cv and in cf / cb
};

// operands of chunk k of the row tile at m0 into stage sb (A hi | B hi | A lo | B lo);
// thread tid forms row tid % 128 for the K quads tid / 128 and tid / 128 + 2, and
// column operand entries tid and tid + 256.  Every load of a thread's entries
// goes out before the first is used (indices clamped into range, padding masked
// afterwards), so that they are in flight together.
__device__ void tc_form(const TetElem& d, const TcSeg& sg, const TcRow& rw, const TcChunk& k, int ncp,
                        const float* tabJ, const float* cv, const float* cfb, const float* vq, const int* fpo,
                        float* sb) {
    const int tid = threadIdx.x, Np = d.Np, Nq = d.Nq, Nc = Np + d.t / M;
    float* Ah = sb;
    float* Bh = Ah + TMT * TKC;
    float* Al = Bh + TNP * TKC;
    float* Bl = Al + TMT * TKC;
    const int rl = tid & (TMT - 1);
    const float sgn = k.vol ? (k.j > 0 ? -1.f : 1.f) : (k.j > 1 ? -1.f : 1.f);
    float va[2][4], vb[2][4];
    // row operand
    if (k.vol) {
        const float* dphi = tabJ + d.vtab + (size_t)Nq * Np + rw.i;
        const float* o = cv + rw.cvo + k.j;
        float g0[2][4], g1[2][4], g2[2][4], c0[2][4], c1[2][4], c2[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = min(k.p0 + 4 * ((tid >> 7) + 2 * h) + u, k.np - 1);
                g0[h][u] = dphi[(size_t)p * Np];
                g1[h][u] = dphi[((size_t)Nq + p) * Np];
                g2[h][u] = dphi[((size_t)2 * Nq + p) * Np];
                const float* op = o + (size_t)p * 300;
                c0[h][u] = op[0];
                c1[h][u] = op[M * 4];
                c2[h][u] = op[2 * M * 4];
            }
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                va[h][u] = sgn * fmaf(g2[h][u], c2[h][u], fmaf(g1[h][u], c1[h][u], g0[h][u] * c0[h][u]));
    } else {
        float rb[2][4], cb4[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = min(k.p0 + 4 * ((tid >> 7) + 2 * h) + u, k.np - 1);
                rb[h][u] = sg.f < 0 ? basis_row_t(tabJ, d, Nq + p)[rw.i]
                                    : tabJ[d.ttab[sg.f] + (size_t)(p - d.soff[sg.f]) * sg.rdiv + rw.i];
                cb4[h][u] = cfb[(size_t)p * 125 + rw.cfo + k.j];
            }
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int u = 0; u < 4; ++u) va[h][u] = sgn * rb[h][u] * cb4[h][u];
    }
    // column operand
    int nn[2], qq[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int it = min(tid + h * NTH, ncp * (TKC / 4) - 1);
        nn[h] = it % ncp;
        qq[h] = it / ncp;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int p = min(k.p0 + 4 * qq[h] + u, k.np - 1), c = min(nn[h], Nc - 1);
            float x;
            if (k.vol) {
                x = k.j == 0 ? tabJ[d.vtab + (size_t)p * Np + min(c, Np - 1)]
                             : vq[((size_t)(k.j - 1) * NPT + p) * NCM + c];
            } else if (k.j == 0) {
                x = basis_row_t(tabJ, d, Nq + p)[min(c, Np - 1)];
            } else if (k.j == 1) {
                const int f = face_of_point(d, p), nf = d.nfp[f];
                const int l = min(max(c - Np - fpo[f], 0), nf - 1);
                x = tabJ[d.ttab[f] + (size_t)(p - d.soff[f]) * nf + l];
            } else {
                x = vq[((size_t)(k.j - 2) * NPT + Nq + p) * NCM + c];
            }
            vb[h][u] = x;
        }
    }
    // masks and stores
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = (tid >> 7) + 2 * h;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (!rw.live || k.p0 + 4 * q + u >= k.np) va[h][u] = 0.f;
        tc_put4(Ah, Al, rl, q, va[h]);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (tid + h * NTH >= ncp * (TKC / 4)) continue;
        const int n = nn[h], q = qq[h];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            bool ok = n < Nc && k.p0 + 4 * q + u < k.np;
            if (ok && k.j == 0) ok = n < Np;
            if (ok && !k.vol && k.j == 1) {
                const int p = k.p0 + 4 * q + u, f = face_of_point(d, p), l = n - Np - fpo[f];
                ok = l >= 0 && l < d.nfp[f];
            }
            if (!ok) vb[h][u] = 0.f;
        }
        tc_put4(Bh, Bl, n, q, vb[h]);
    }
    asm volatile("fence.proxy.async.shared::cta;");
}

// wait for the batch committed to stage sb (if any); on a timeout the status
// records it and the tile's results are not stored
__device__ __forceinline__ void tc_wait(TcState& ts, uint32_t& pending, int sb, bool& ok, int* sflag) {
    if (!((pending >> sb) & 1u)) return;
    const uint32_t bar = ts.bar + 8u * sb, par = (ts.phase >> sb) & 1u;
    if (!mbar_wait_bounded(bar, par, 1 << 24)) {
        ok = false;
        if (threadIdx.x == 0) atomicOr(sflag, 4);
        mbar_wait_bounded(bar, par, 1 << 24);
    }
    ts.phase ^= 1u << sb;
    pending &= ~(1u << sb);
}

// One 128-row tile of a 3xTF32 product into tensor memory: nch chunks, chunk ci
// formed by form(ci, stage) into A hi | B hi | A lo | B lo (K-major core
// matrices), N = ncp columns; the threads form chunk c + 1 while the tensor
// cores run chunk c.  Returns false when a wait timed out (nothing to store).
template <class Form>
__device__ bool tc_tile(TcState& ts, float* st0, int nch, int ncp, Form&& form, int* sflag) {
    const int tid = threadIdx.x;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(ncp >> 3) << 17) |
                           ((uint32_t)(TMT >> 4) << 24);
    uint32_t pending = 0;
    bool ok = true;
    form(0, st0);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    for (int ci = 0; ci < nch; ++ci) {
        const int sbi = ci & 1;
        if (tid == 0) {
            const float* Ah = st0 + sbi * TSTAGE;
            const float* Bh = Ah + TMT * TKC;
            const float* Al = Bh + TNP * TKC;
            const float* Bl = Al + TMT * TKC;
            for (int s = 0; s < TKC / 8; ++s) {
                const uint32_t off = s * 256;
                const uint64_t ah = umma_desc(smem_u32(Ah) + off, 128, (TKC / 4) * 128);
                const uint64_t bh = umma_desc(smem_u32(Bh) + off, 128, (TKC / 4) * 128);
                const uint64_t al = umma_desc(smem_u32(Al) + off, 128, (TKC / 4) * 128);
                const uint64_t bl = umma_desc(smem_u32(Bl) + off, 128, (TKC / 4) * 128);
                const uint32_t acc = (ci > 0 || s > 0) ? 1u : 0u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                             :: "r"(ts.tmem), "l"(ah), "l"(bh), "r"(idesc), "r"(acc));
                asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;"
                             :: "r"(ts.tmem), "l"(ah), "l"(bl), "r"(idesc));
                asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;"
                             :: "r"(ts.tmem), "l"(al), "l"(bh), "r"(idesc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(ts.bar + 8u * sbi));
        }
        pending |= 1u << sbi;
        if (ci + 1 < nch) {
            tc_wait(ts, pending, sbi ^ 1, ok, sflag);               // the previous batch read the other stage
            if (__syncthreads_or(ok ? 0 : 1)) {
                ok = false;
                break;
            }
            form(ci + 1, st0 + (sbi ^ 1) * TSTAGE);
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
        }
    }
    tc_wait(ts, pending, 0, ok, sflag);
    tc_wait(ts, pending, 1, ok, sflag);
    ok = !__syncthreads_or(ok ? 0 : 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    return ok;
}

// Read a finished tile from tensor memory: store(row of the tile, first column,
// 16 values) for every 16 columns below ncp; warp w reads lanes 32 (w % 4) ..
// + 31, warps 4..7 the second half of the columns.  Ends with the barrier after
// which the next tile may overwrite the accumulator.
template <class Store>
__device__ void tc_tile_store(const TcState& ts, int ncp, Store&& store) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lg = warp & 3, half = warp >> 2;
    const int hc = ((ncp / 2) + 15) / 16 * 16;
    for (int c0 = half * hc; c0 < min(ncp, (half + 1) * hc); c0 += 16) {
        uint32_t v[16];
        const uint32_t addr = ts.tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)c0;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                       "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                       "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                     : "r"(addr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        store(lg * 32 + lane, c0, v);
    }
}

__device__ __forceinline__ void tc_tile_done() {
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
}

// the whole contraction of one element (element rows, then the trace rows of
// each face) into the bordered matrix Mx, FP64 storage
__device__ void contract_tc(const TetElem& d, const float* tabJ, const float* cv, const float* cf, const float* cb,
                            const float* vq, const int* fpo, double* Mx, float* st0, TcState& ts, int* sflag) {
    const int tid = threadIdx.x;
    const int Np = d.Np, LD = d.LD, NU = d.NU, Nc = Np + d.t / M;
    const int ncp = (Nc + 15) / 16 * 16;
    for (int sgi = -1; sgi < 4; ++sgi) {
        TcSeg sg;
        sg.f = sgi;
        sg.rdiv = sgi < 0 ? Np : d.nfp[sgi];
        sg.rows = M * M * sg.rdiv;
        sg.cv = (d.Nq + TKC - 1) / TKC;
        sg.cf = ((sgi < 0 ? d.sfq : d.nfq[sgi]) + TKC - 1) / TKC;
        sg.nch = (sgi < 0 ? 4 * sg.cv : 0) + 5 * sg.cf;
        const float* cfb = sgi < 0 ? cf : cb;
        for (int m0 = 0; m0 < sg.rows; m0 += TMT) {
            TcRow rw;
            {
                const int r = m0 + (tid & (TMT - 1));
                const int ab = r / sg.rdiv, a = ab / M, b = ab - a * M;
                rw.live = r < sg.rows;
                rw.i = rw.live ? r - ab * sg.rdiv : 0;
                rw.cvo = rw.live ? (a * 3 * M + b) * 4 : 0;
                rw.cfo = rw.live ? (a * M + b) * 5 : 0;
            }
            auto form = [&](int ci, float* sb) {
                tc_form(d, sg, rw, tc_chunk(d, sg, ci), ncp, tabJ, cv, cfb, vq, fpo, sb);
            };
            if (tc_tile(ts, st0, sg.nch, ncp, form, sflag)) {
                tc_tile_store(ts, ncp, [&](int rl, int c0, const uint32_t* v) {
                    const int r = m0 + rl;
                    if (r >= sg.rows) return;
                    const int ab = r / sg.rdiv, i = r - ab * sg.rdiv, a = ab / M, b = ab - a * M;
                    const int64_t row = sgi < 0 ? (int64_t)a * Np + i : (int64_t)NU + d.toff[sgi] + a * sg.rdiv + i;
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        const int c = c0 + jj;
                        if (c < Nc) Mx[row * LD + bcol(d, b, c)] = (double)__uint_as_float(v[jj]);
                    }
                });
            }
            tc_tile_done();
        }
    }
}

// The trace rows' Schur product of the mixed form on the tensor cores:
// S = Dt - W Z with W = Wt^T ([n_u][t], trace rows contiguous) and Z ([n_u][t]),
// 3xTF32 as the contraction; tiles of 128 trace rows x 96 trace columns.
__device__ void schur_tc(double* Mx, int NU, int t, int LD, const float* Wt, const float* Zf, float* st0,
                         TcState& ts, int* sflag) {
    const int tid = threadIdx.x;
    const int nch = (NU + TKC - 1) / TKC;
    for (int m0 = 0; m0 < t; m0 += TMT)
        for (int n0 = 0; n0 < t; n0 += TNP) {
            const int nc = min(TNP, t - n0), ncp = (nc + 15) / 16 * 16;
            auto form = [&](int ci, float* sb) {
                float* Ah = sb;
                float* Bh = Ah + TMT * TKC;
                float* Al = Bh + TNP * TKC;
                float* Bl = Al + TMT * TKC;
                const int k0 = ci * TKC, rl = tid & (TMT - 1), r = min(m0 + rl, t - 1);
                const bool live = m0 + rl < t;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int q = (tid >> 7) + 2 * h;
                    float v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) v[u] = Wt[(size_t)min(k0 + 4 * q + u, NU - 1) * t + r];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (!live || k0 + 4 * q + u >= NU) v[u] = 0.f;
                    tc_put4(Ah, Al, rl, q, v);
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int it = tid + h * NTH;
                    if (it >= ncp * (TKC / 4)) continue;
                    const int n = it % ncp, q = it / ncp, c = n0 + min(n, nc - 1);
                    float v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) v[u] = Zf[(size_t)min(k0 + 4 * q + u, NU - 1) * t + c];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (n >= nc || k0 + 4 * q + u >= NU) v[u] = 0.f;
                    tc_put4(Bh, Bl, n, q, v);
                }
                asm volatile("fence.proxy.async.shared::cta;");
            };
            if (tc_tile(ts, st0, nch, ncp, form, sflag)) {
                tc_tile_store(ts, ncp, [&](int rl, int c0, const uint32_t* v) {
                    const int r = m0 + rl;
                    if (r >= t) return;
                    double* row = Mx + (size_t)(NU + r) * LD + NU + n0;
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj)
                        if (c0 + jj < nc) row[c0 + jj] -= (double)__uint_as_float(v[jj]);
                });
            }
            tc_tile_done();
        }
}

// Trace rows of the mixed form, after the FP64 LU of the interior block At
// (partial pivoting, panels of NB columns; the interchanges of a panel are
// recorded in gpiv and applied only to the columns right of it inside At, so
// the L of each panel is stored at that panel's row order):
//  * z = L^{-1} P Rt in FP64 and Z = L^{-1} P Bt in FP32, panel by panel: the
//    panel's interchanges, then its unit-lower block and the update of the rows
//    below, one thread per column with the panel's values in registers;
//  * W = Ct U^{-1} in FP32, panel by panel over the columns of U (W kept
//    transposed so that threads over trace rows read consecutive words);
//  * Z back into the bordered matrix (the recovery reads it), the right-hand
//    side Rh - W z in FP64 and S = Dt - W Z on the tensor cores (3xTF32).
template <int NB>
__device__ void trace_schur_f32(double* Mx, int NU, int t, int LD, const int* gpiv, float* Wt, float* Zf,
                                float* smf, TcState& ts, int* sflag) {
    const int tid = threadIdx.x, NR = NU + t;
    for (int idx = tid; idx < NU * t; idx += NTH) {
        const int i = idx / t, r = idx - i * t;
        Wt[idx] = (float)Mx[(size_t)(NU + r) * LD + i];
        Zf[idx] = (float)Mx[(size_t)i * LD + NU + r];
    }
    __syncthreads();
    // Z = L^{-1} P Bt (FP32, one thread per column) and z = L^{-1} P Rt (FP64:
    // interchanges and the panel's block by one thread, the rows below by all)
    constexpr int TPS = 304;                            // row stride of a staged panel (t <= 300)
    float* sL = smf;                                    // [NU - k0][NB] panel of L
    float* sZp = smf + M * NPMAX * NB;                  // [NB][TPS] the panel's rows of Z
    __shared__ double zp[NB];
    double* zc = Mx + NR;                               // column NR, stride LD
    for (int k0 = 0; k0 < NU; k0 += NB) {
        const int kb = min(NB, NU - k0);
        for (int idx = tid; idx < (NU - k0) * NB; idx += NTH) {
            const int i = idx / NB, j = idx - i * NB;
            sL[idx] = j < kb ? (float)Mx[(size_t)(k0 + i) * LD + k0 + j] : 0.0f;
        }
        __syncthreads();
        for (int r = tid; r < t; r += NTH) {
            float* zf = Zf + r;
            for (int j = 0; j < kb; ++j) {
                const int pr = gpiv[k0 + j];
                if (pr != k0 + j) {
                    const float x = zf[(size_t)(k0 + j) * t];
                    zf[(size_t)(k0 + j) * t] = zf[(size_t)pr * t];
                    zf[(size_t)pr * t] = x;
                }
            }
            float zv[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) zv[j] = j < kb ? zf[(size_t)(k0 + j) * t] : 0.0f;
#pragma unroll
            for (int j = 0; j < NB; ++j)
#pragma unroll
                for (int jj = j + 1; jj < NB; ++jj)
                    if (jj < kb) zv[jj] = fmaf(-sL[jj * NB + j], zv[j], zv[jj]);
#pragma unroll
            for (int j = 0; j < NB; ++j)
                if (j < kb) zf[(size_t)(k0 + j) * t] = zv[j];
        }
        if (tid == NTH - 1) {
            for (int j = 0; j < kb; ++j) {
                const int pr = gpiv[k0 + j];
                if (pr != k0 + j) {
                    const double x = zc[(size_t)(k0 + j) * LD];
                    zc[(size_t)(k0 + j) * LD] = zc[(size_t)pr * LD];
                    zc[(size_t)pr * LD] = x;
                }
            }
            for (int j = 0; j < kb; ++j) {
                double zj = zc[(size_t)(k0 + j) * LD];
                for (int i = 0; i < j; ++i) zj -= Mx[(size_t)(k0 + j) * LD + k0 + i] * zp[i];
                zp[j] = zj;
                zc[(size_t)(k0 + j) * LD] = zj;
            }
        }
        __syncthreads();
        for (int idx = tid; idx < kb * t; idx += NTH) {          // the panel's rows of Z, for the update
            const int j = idx / t, r = idx - j * t;
            sZp[j * TPS + r] = Zf[(size_t)(k0 + j) * t + r];
        }
        for (int i = k0 + kb + tid; i < NU; i += NTH) {
            double s2 = zc[(size_t)i * LD];
            for (int j = 0; j < kb; ++j) s2 -= Mx[(size_t)i * LD + k0 + j] * zp[j];
            zc[(size_t)i * LD] = s2;
        }
        __syncthreads();
        // rows below the panel: Z_below -= L_panel Z_panel in 4 x 4 register tiles
        {
            const int i0 = k0 + kb, nr = NU - i0, nrt = (nr + 3) / 4, nct = (t + 3) / 4;
            for (int tile = tid; tile < nrt * nct; tile += NTH) {
                const int ti = tile / nct, tc = tile - ti * nct, ib = i0 + 4 * ti, cb = 4 * tc;
                float acc[4][4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        acc[u][v] = Zf[(size_t)min(ib + u, NU - 1) * t + min(cb + v, t - 1)];
                for (int j = 0; j < kb; ++j) {
                    float l[4], z[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) l[u] = sL[(size_t)(min(ib + u, NU - 1) - k0) * NB + j];
#pragma unroll
                    for (int v = 0; v < 4; ++v) z[v] = sZp[j * TPS + min(cb + v, t - 1)];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(-l[u], z[v], acc[u][v]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        if (ib + u < NU && cb + v < t) Zf[(size_t)(ib + u) * t + cb + v] = acc[u][v];
            }
        }
        __syncthreads();
    }
    // W = Ct U^{-1}: W U = Ct, panel by panel over the columns of U
    float* sUp = smf;                                   // [NB][NU - k0] panel rows of U
    float* sDi = smf + NB * NU;                         // [NB] reciprocal diagonal
    float* sWp = smf + M * NPMAX * NB + NB;             // [NB][TPS] the panel's columns of W
    for (int k0 = 0; k0 < NU; k0 += NB) {
        const int kb = min(NB, NU - k0), w = NU - k0;
        for (int idx = tid; idx < NB * w; idx += NTH) {
            const int j = idx / w, c = idx - j * w;
            sUp[idx] = (j < kb && c >= j) ? (float)Mx[(size_t)(k0 + j) * LD + k0 + c] : 0.0f;
        }
        if (tid < NB) {
            const float u = tid < kb ? (float)Mx[(size_t)(k0 + tid) * LD + k0 + tid] : 1.0f;
            sDi[tid] = u != 0.0f ? 1.0f / u : 1.0f;
        }
        __syncthreads();
        for (int r = tid; r < t; r += NTH) {
            float* wc = Wt + r;
            float wv[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) wv[j] = j < kb ? wc[(size_t)(k0 + j) * t] : 0.0f;
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                if (j >= kb) continue;
#pragma unroll
                for (int i = 0; i < j; ++i) wv[j] = fmaf(-wv[i], sUp[i * w + j], wv[j]);
                wv[j] *= sDi[j];
            }
#pragma unroll
            for (int j = 0; j < NB; ++j)
                if (j < kb) {
                    wc[(size_t)(k0 + j) * t] = wv[j];
                    sWp[j * TPS + r] = wv[j];
                }
        }
        __syncthreads();
        // columns right of the panel: W_right -= W_panel U_panel,right in 4 x 4 register tiles
        // (W kept transposed: row c of Wt is column c of W)
        {
            const int c0 = kb, nw = w - kb, nrt = (nw + 3) / 4, nct = (t + 3) / 4;
            for (int tile = tid; tile < nrt * nct; tile += NTH) {
                const int ti = tile / nct, tc = tile - ti * nct, cc = c0 + 4 * ti, rb = 4 * tc;
                float acc[4][4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        acc[u][v] = Wt[(size_t)(k0 + min(cc + u, w - 1)) * t + min(rb + v, t - 1)];
                for (int j = 0; j < kb; ++j) {
                    float uu[4], wr[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) uu[u] = sUp[j * w + min(cc + u, w - 1)];
#pragma unroll
                    for (int v = 0; v < 4; ++v) wr[v] = sWp[j * TPS + min(rb + v, t - 1)];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(-uu[u], wr[v], acc[u][v]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        if (cc + u < w && rb + v < t) Wt[(size_t)(k0 + cc + u) * t + rb + v] = acc[u][v];
            }
        }
        __syncthreads();
    }
    // Z to the bordered matrix (FP32 values in FP64 storage)
    for (int idx = tid; idx < NU * t; idx += NTH) {
        const int i = idx / t, r = idx - i * t;
        Mx[(size_t)i * LD + NU + r] = (double)Zf[idx];
    }
    // right-hand side of the trace rows: Rh - W z (FP64)
    for (int r = tid; r < t; r += NTH) {
        double s2 = Mx[(size_t)(NU + r) * LD + NR];
        for (int i = 0; i < NU; ++i) s2 -= (double)Wt[(size_t)i * t + r] * Mx[(size_t)i * LD + NR];
        Mx[(size_t)(NU + r) * LD + NR] = s2;
    }
    // S = Dt - W Z on the tensor cores
    __syncthreads();
    schur_tc(Mx, NU, t, LD, Wt, Zf, smf, ts, sflag);
}

// TJ: type of the Jacobian coefficients, the column variations and the
// contraction (double: FP64 form; float: mixed form).  Pointwise terms, lifting
// operators, mass term, right-hand side and the elimination are FP64 in both.
template <class TJ, int NBE>
__device__ void process_element(const KArgs& A, const TetElem& d, double* W, double* sm, int* sflag, TcState* ts) {
    const int tid = threadIdx.x;
    const int Np = d.Np, Nq = d.Nq, NU = d.NU, t = d.t, LD = d.LD, sfq = d.sfq;
    const int sfp = t / M, Nc = Np + sfp, npt = Nq + sfq;
    const double* phi = A.tab + d.vtab;
    const double* dphi = phi + (size_t)Nq * Np;
    double* Mx = A.mat + d.moff;
    double* Gk = A.rec + d.roff;                     // [3][Np][Np]
    double* Hk = Gk + 3 * Np * Np;                   // [3][Np][sfp]
    double* dq0 = Hk + 3 * Np * sfp;                 // [3][m][Np]
    double* sU = sm + S_U;
    double* sUs = sm + S_US;
    double* sQ = sm + S_Q;
    double* sQL = sm + S_QL;
    double* sUH = sm + S_UH;
    double* sD = sm + S_DYN;
    double* gv = W + W_GV;
    double* gf = W + W_GF;
    int fpo[4];
    fpo[0] = 0;
    for (int f = 1; f < 4; ++f) fpo[f] = fpo[f - 1] + d.nfp[f - 1];

    gather_element(A, d, sm);
    load_geometry(A, d, gv, gf);
    __syncthreads();
    // physical gradients at the volume points and the basis values, both times the
    // point weight w|J| (so that E and M take one multiply-add per point), mass matrix
    double* dp = W + W_DP;                               // [Nq][3][NPMAX] w|J| grad phi_i
    double* wphi = W + W_VQ;                             // [Nq][NPMAX] w|J| phi_i (free until psi/chi)
    for (int idx = tid; idx < Nq * Np; idx += NTH) {
        const int g = idx / Np, i = idx - g * Np;
        const double* Ji = gv + g * 10 + 1;
        const double d0 = dphi[(size_t)g * Np + i], d1 = dphi[((size_t)Nq + g) * Np + i],
                     d2 = dphi[((size_t)2 * Nq + g) * Np + i];
        for (int k = 0; k < 3; ++k)
            dp[(g * 3 + k) * NPMAX + i] = gv[g * 10] * (Ji[0 * 3 + k] * d0 + Ji[1 * 3 + k] * d1 + Ji[2 * 3 + k] * d2);
        wphi[g * NPMAX + i] = gv[g * 10] * phi[(size_t)g * Np + i];
    }
    __syncthreads();
    double* Mm = W + W_MM;
    for (int idx = tid; idx < Np * Np; idx += NTH) {
        const int i = idx / Np, j = idx - i * Np;
        double s = 0.0;
        for (int g = 0; g < Nq; ++g) s += wphi[g * NPMAX + i] * phi[(size_t)g * Np + j];
        Mm[i * NPMAX + j] = s;
    }
    // E_k = (phi_j, d_k phi_i) into G; B_q,k = -<phi_i mu_l n_k> into H
    for (int idx = tid; idx < 3 * Np * Np; idx += NTH) {
        const int k = idx / (Np * Np), rem = idx - k * Np * Np, i = rem / Np, j = rem - i * Np;
        double s = 0.0;
        for (int g = 0; g < Nq; ++g) s += dp[(g * 3 + k) * NPMAX + i] * phi[(size_t)g * Np + j];
        Gk[idx] = s;
    }
    for (int idx = tid; idx < 3 * Np * sfp; idx += NTH) {
        const int k = idx / (Np * sfp), rem = idx - k * Np * sfp, i = rem / sfp, cp = rem - i * sfp;
        int f = 0, l = cp;
        while (f < 3 && l >= d.nfp[f]) { l -= d.nfp[f]; ++f; }
        const double* phf = A.tab + d.ftab[f];
        const double* mu = A.tab + d.ttab[f];
        double s = 0.0;
        for (int q = 0; q < d.nfq[f]; ++q)
            s += gf[(d.soff[f] + q) * 3 + k] * phf[(size_t)q * Np + i] * mu[(size_t)q * d.nfp[f] + l];
        Hk[idx] = -s;
    }
    __syncthreads();
    // Cholesky factor of the mass matrix (one warp)
    if (tid < 32) {
        for (int j = 0; j < Np; ++j) {
            if (tid == 0) {
                double s = Mm[j * NPMAX + j];
                for (int k = 0; k < j; ++k) s -= Mm[j * NPMAX + k] * Mm[j * NPMAX + k];
                Mm[j * NPMAX + j] = s > 0.0 ? sqrt(s) : 1.0;
                if (!(s > 0.0)) atomicOr(sflag, 1);
            }
            __syncwarp();
            const double ljj = Mm[j * NPMAX + j];
            for (int i = j + 1 + tid; i < Np; i += 32) {
                double s = Mm[i * NPMAX + j];
                for (int k = 0; k < j; ++k) s -= Mm[i * NPMAX + k] * Mm[j * NPMAX + k];
                Mm[i * NPMAX + j] = s / ljj;
            }
            __syncwarp();
        }
    }
    __syncthreads();
    // G_k = M^{-1} E_k, H_k = M^{-1} B_q,k: one column per thread (forward, backward substitution)
    for (int col = tid; col < 3 * Nc; col += NTH) {
        const int k = col / Nc, c = col - k * Nc;
        double* x;
        int st;
        if (c < Np) { x = Gk + (size_t)k * Np * Np + c; st = Np; }
        else { x = Hk + (size_t)k * Np * sfp + (c - Np); st = sfp; }
        for (int i = 0; i < Np; ++i) {
            double s = x[i * st];
            for (int j = 0; j < i; ++j) s -= Mm[i * NPMAX + j] * x[j * st];
            x[i * st] = s / Mm[i * NPMAX + i];
        }
        for (int i = Np - 1; i >= 0; --i) {
            double s = x[i * st];
            for (int j = i + 1; j < Np; ++j) s -= Mm[j * NPMAX + i] * x[j * st];
            x[i * st] = s / Mm[i * NPMAX + i];
        }
    }
    __syncthreads();
    // lifted gradient Q_lift = -G U - H Uhat (the gradient equations hold exactly)
    for (int idx = tid; idx < 3 * NU; idx += NTH) {
        const int k = idx / NU, rem = idx - k * NU, a = rem / Np, i = rem - a * Np;
        double s = 0.0;
        for (int j = 0; j < Np; ++j) s += Gk[((size_t)k * Np + i) * Np + j] * sU[a * Np + j];
        for (int f = 0; f < 4; ++f)
            for (int l = 0; l < d.nfp[f]; ++l)
                s += Hk[((size_t)k * Np + i) * sfp + fpo[f] + l] * sUH[d.toff[f] + a * d.nfp[f] + l];
        sQL[idx] = -s;
        dq0[idx] = -s - sQ[idx];
    }
    __syncthreads();
    // values at the points; psi | chi (the q variation of unit U / Uhat columns)
    double* pu = W + W_PU;
    double* pq = W + W_PQ;
    double* pl = W + W_PL;
    double* ph = W + W_PH;
    for (int x = tid; x < npt; x += NTH) {
        const double* br = basis_row(A, d, x);
        double u[M], q[M][3], ql[M][3];
        for (int a = 0; a < M; ++a) { u[a] = 0.0; for (int k = 0; k < 3; ++k) { q[a][k] = 0.0; ql[a][k] = 0.0; } }
        for (int j = 0; j < Np; ++j) {
            const double w = br[j];
            for (int a = 0; a < M; ++a) {
                u[a] += w * sU[a * Np + j];
                for (int k = 0; k < 3; ++k) {
                    q[a][k] += w * sQ[(k * M + a) * Np + j];
                    ql[a][k] += w * sQL[(k * M + a) * Np + j];
                }
            }
        }
        for (int a = 0; a < M; ++a) {
            pu[x * M + a] = u[a];
            for (int k = 0; k < 3; ++k) { pq[(x * M + a) * 3 + k] = q[a][k]; pl[(x * M + a) * 3 + k] = ql[a][k]; }
        }
        if (x >= Nq) {
            const int r = x - Nq, f = face_of_point(d, r), s = r - d.soff[f];
            const double* mu = A.tab + d.ttab[f] + (size_t)s * d.nfp[f];
            for (int a = 0; a < M; ++a) {
                double v = 0.0;
                for (int l = 0; l < d.nfp[f]; ++l) v += mu[l] * sUH[d.toff[f] + a * d.nfp[f] + l];
                ph[r * M + a] = v;
            }
        }
    }
    const TJ* tabJ = jtab<TJ>(A);
    const TJ* GJ;
    const TJ* HJ;
    if constexpr (sizeof(TJ) == sizeof(double)) {
        GJ = reinterpret_cast<const TJ*>(Gk);
        HJ = reinterpret_cast<const TJ*>(Hk);
    } else {
        TJ* gh = reinterpret_cast<TJ*>(W + W_GHF);
        for (int i = tid; i < 3 * Np * (Np + sfp); i += NTH) gh[i] = (TJ)Gk[i];   // G and H are contiguous
        GJ = gh;
        HJ = gh + 3 * Np * Np;
        __syncthreads();
    }
    TJ* vq = reinterpret_cast<TJ*>(W + W_VQ);
    const int nc4 = (Nc + 3) / 4;                       // four columns per thread: one basis load per 4 FMAs
    for (int idx = tid; idx < 3 * npt * nc4; idx += NTH) {
        const int k = idx / (npt * nc4), rem = idx - k * npt * nc4, x = rem / nc4, c0 = 4 * (rem - x * nc4);
        const TJ* br = basis_row_t(tabJ, d, x);
        const TJ* gp[4];
        int st[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = min(c0 + u, Nc - 1);
            if (c < Np) { gp[u] = GJ + (size_t)k * Np * Np + c; st[u] = Np; }
            else { gp[u] = HJ + (size_t)k * Np * sfp + (c - Np); st[u] = sfp; }
        }
        TJ s[4] = {0, 0, 0, 0};
        for (int j = 0; j < Np; ++j) {
            const TJ b = br[j];
#pragma unroll
            for (int u = 0; u < 4; ++u) s[u] += b * gp[u][j * st[u]];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (c0 + u < Nc) vq[((size_t)k * NPT + x) * NCM + c0 + u] = s[u];
    }
    __syncthreads();
    // A1: fluxes and their Jacobians at the points
    const PhysT<double>& P = A.ph;
    using SJ = std::conditional_t<sizeof(TJ) == sizeof(float), float, double>;   // Jacobian terms' type
    TJ* cv = reinterpret_cast<TJ*>(W + W_CV);
    TJ* cf = reinterpret_cast<TJ*>(W + W_CF);
    TJ* cb = reinterpret_cast<TJ*>(W + W_CB);
    double* rv = W + W_RV;
    double* rf = W + W_RF;
    double* rb = W + W_RB;
    for (int x = tid; x < npt; x += NTH) {
        double u[M], q[M][3], ql[M][3];
        for (int a = 0; a < M; ++a) {
            u[a] = pu[x * M + a];
            for (int k = 0; k < 3; ++k) { q[a][k] = pq[(x * M + a) * 3 + k]; ql[a][k] = pl[(x * M + a) * 3 + k]; }
        }
        if (x < Nq) {
            const double* g = gv + x * 10;
            const double wJ = -A.dt * g[0];
            const double* Ji = g + 1;
            double Fc[M][3], Fv[M][3];
            conv_flux<3, double, double>(u, P, Fc);
            visc_flux<3, double, double>(u, ql, 0.0, P, Fv);
            for (int a = 0; a < M; ++a)
                for (int r = 0; r < 3; ++r) {
                    double s = 0.0;
                    for (int k = 0; k < 3; ++k) s += Ji[r * 3 + k] * (Fc[a][k] - Fv[a][k]);
                    rv[(x * M + a) * 3 + r] = wJ * s;
                }
            if constexpr (sizeof(TJ) == sizeof(float)) {
                // Jacobian coefficients in the contraction's precision (FP32 in the mixed form)
                TJ* o = cv + (size_t)x * 300;
                const PhysT<SJ>& PJ = jphys<SJ>(A);
                SJ us[M], qs[M][3], Js[9];
                for (int a = 0; a < M; ++a) { us[a] = (SJ)u[a]; for (int k = 0; k < 3; ++k) qs[a][k] = (SJ)q[a][k]; }
                for (int k = 0; k < 9; ++k) Js[k] = (SJ)Ji[k];
                const SJ wJs = (SJ)wJ;
                for (int b = 0; b < M; ++b) {
                    DirT<SJ> ud[M];
                    for (int a = 0; a < M; ++a) ud[a] = {us[a], a == b ? SJ(1) : SJ(0)};
                    DirT<SJ> Fcd[M][3], Fvd[M][3];
                    conv_flux<3, DirT<SJ>, SJ>(ud, PJ, Fcd);
                    visc_flux<3, DirT<SJ>, SJ>(ud, qs, SJ(0), PJ, Fvd);
                    for (int a = 0; a < M; ++a)
                        for (int r = 0; r < 3; ++r) {
                            SJ s = SJ(0);
                            for (int k = 0; k < 3; ++k) s += Js[r * 3 + k] * (Fcd[a][k].t - Fvd[a][k].t);
                            o[((a * 3 + r) * M + b) * 4 + 0] = (TJ)(wJs * s);
                        }
                    for (int l = 0; l < 3; ++l) {
                        SJ qe[M][3];
                        for (int a = 0; a < M; ++a) for (int k = 0; k < 3; ++k) qe[a][k] = (a == b && k == l) ? SJ(1) : SJ(0);
                        SJ Fq[M][3];
                        visc_flux<3, SJ, SJ>(us, qe, SJ(0), PJ, Fq);
                        for (int a = 0; a < M; ++a)
                            for (int r = 0; r < 3; ++r) {
                                SJ s = SJ(0);
                                for (int k = 0; k < 3; ++k) s += Js[r * 3 + k] * Fq[a][k];
                                o[((a * 3 + r) * M + b) * 4 + 1 + l] = (TJ)(-wJs * s);
                            }
                    }
                }
            } else {
                TJ* o = cv + (size_t)x * 300;
                for (int b = 0; b < M; ++b) {
                    Dir ud[M];
                    for (int a = 0; a < M; ++a) ud[a] = {u[a], a == b ? 1.0 : 0.0};
                    Dir Fcd[M][3], Fvd[M][3];
                    conv_flux<3, Dir, double>(ud, P, Fcd);
                    visc_flux<3, Dir, double>(ud, q, 0.0, P, Fvd);
                    for (int a = 0; a < M; ++a)
                        for (int r = 0; r < 3; ++r) {
                            double s = 0.0;
                            for (int k = 0; k < 3; ++k) s += Ji[r * 3 + k] * (Fcd[a][k].t - Fvd[a][k].t);
                            o[((a * 3 + r) * M + b) * 4 + 0] = (TJ)(wJ * s);
                        }
                    for (int l = 0; l < 3; ++l) {
                        double qe[M][3];
                        for (int a = 0; a < M; ++a) for (int k = 0; k < 3; ++k) qe[a][k] = (a == b && k == l) ? 1.0 : 0.0;
                        double Fq[M][3];
                        visc_flux<3, double, double>(u, qe, 0.0, P, Fq);
                        for (int a = 0; a < M; ++a)
                            for (int r = 0; r < 3; ++r) {
                                double s = 0.0;
                                for (int k = 0; k < 3; ++k) s += Ji[r * 3 + k] * Fq[a][k];
                                o[((a * 3 + r) * M + b) * 4 + 1 + l] = (TJ)(-wJ * s);
                            }
                    }
                }
            }
        } else {
            const int r = x - Nq, f = face_of_point(d, r), tag = d.tag[f];
            const double* nw = gf + r * 3;
            const double nrm = sqrt(nw[0] * nw[0] + nw[1] * nw[1] + nw[2] * nw[2]);
            double uh[M];
            for (int a = 0; a < M; ++a) uh[a] = ph[r * M + a];
            const double nh[3] = {nw[0] / nrm, nw[1] / nrm, nw[2] / nrm};
            const double taun = nrm * (A.tau_mode ? stab_tau<3, double, double>(uh, nh, d.hinv, P) : A.tau);
            double Fc[M][3], Fv[M][3];
            conv_flux<3, double, double>(uh, P, Fc);
            visc_flux<3, double, double>(uh, ql, 0.0, P, Fv);
            for (int a = 0; a < M; ++a) {
                double fn = 0.0;
                for (int k = 0; k < 3; ++k) fn += (Fc[a][k] - Fv[a][k]) * nw[k];
                const double fh = fn + taun * (u[a] - uh[a]);
                rf[r * M + a] = A.dt * fh;
                const double ub_a = tag == 1 ? A.ub[a] : 0.0;
                rb[r * M + a] = boundary_form<M>(tag, a, fh, nrm, u, uh, ub_a, A.ew);
            }
            TJ* of = cf + (size_t)r * 125;
            TJ* ob = cb + (size_t)r * 125;
            // element rows take dt * dfhat; trace rows dfhat on flux rows, the algebraic forms
            // otherwise (tag 1 uhat - u_b, tag 2 uhat - u, tags 3 / 4 uhat_v, and on isothermal
            // walls uhat_rhoE - uhat_rho e_w)
            auto put = [&](int a, int b, int kind, double v) {
                of[(a * M + b) * 5 + kind] = (TJ)(A.dt * v);
                double w = v;
                if (!boundary_row_is_flux<M>(tag, a)) {
                    w = 0.0;
                    if (kind == 1 && a == b) w = nrm;
                    if (tag == 2 && kind == 0 && a == b) w = -nrm;
                    if (tag == 3 && a == M - 1 && kind == 1 && b == 0) w = -nrm * A.ew;
                }
                ob[(a * M + b) * 5 + kind] = (TJ)w;
            };
            if constexpr (sizeof(TJ) == sizeof(float)) {
                const PhysT<SJ>& PJ = jphys<SJ>(A);
                SJ uhs[M], qs[M][3], nws[3], nhs[3];
                for (int a = 0; a < M; ++a) { uhs[a] = (SJ)uh[a]; for (int k = 0; k < 3; ++k) qs[a][k] = (SJ)q[a][k]; }
                for (int k = 0; k < 3; ++k) { nws[k] = (SJ)nw[k]; nhs[k] = (SJ)nh[k]; }
                for (int b = 0; b < M; ++b) {
                    DirT<SJ> ud[M];
                    for (int a = 0; a < M; ++a) ud[a] = {uhs[a], a == b ? SJ(1) : SJ(0)};
                    DirT<SJ> Fcd[M][3], Fvd[M][3];
                    conv_flux<3, DirT<SJ>, SJ>(ud, PJ, Fcd);
                    visc_flux<3, DirT<SJ>, SJ>(ud, qs, SJ(0), PJ, Fvd);
                    const double dtau =
                        A.tau_mode ? nrm * (double)stab_tau<3, DirT<SJ>, SJ>(ud, nhs, (SJ)d.hinv, PJ).t : 0.0;
                    for (int a = 0; a < M; ++a) {
                        SJ fn = SJ(0);
                        for (int k = 0; k < 3; ++k) fn += (Fcd[a][k].t - Fvd[a][k].t) * nws[k];
                        put(a, b, 0, a == b ? taun : 0.0);
                        put(a, b, 1, (double)fn - (a == b ? taun : 0.0) + (u[a] - uh[a]) * dtau);
                    }
                    for (int l = 0; l < 3; ++l) {
                        SJ qe[M][3];
                        for (int a = 0; a < M; ++a) for (int k = 0; k < 3; ++k) qe[a][k] = (a == b && k == l) ? SJ(1) : SJ(0);
                        SJ Fq[M][3];
                        visc_flux<3, SJ, SJ>(uhs, qe, SJ(0), PJ, Fq);
                        for (int a = 0; a < M; ++a) {
                            SJ fn = SJ(0);
                            for (int k = 0; k < 3; ++k) fn += Fq[a][k] * nws[k];
                            put(a, b, 2 + l, -(double)fn);
                        }
                    }
                }
            } else {
                for (int b = 0; b < M; ++b) {
                    Dir ud[M];
                    for (int a = 0; a < M; ++a) ud[a] = {uh[a], a == b ? 1.0 : 0.0};
                    Dir Fcd[M][3], Fvd[M][3];
                    conv_flux<3, Dir, double>(ud, P, Fcd);
                    visc_flux<3, Dir, double>(ud, q, 0.0, P, Fvd);
                    const double dtau = A.tau_mode ? nrm * stab_tau<3, Dir, double>(ud, nh, d.hinv, P).t : 0.0;
                    for (int a = 0; a < M; ++a) {
                        double fn = 0.0;
                        for (int k = 0; k < 3; ++k) fn += (Fcd[a][k].t - Fvd[a][k].t) * nw[k];
                        put(a, b, 0, a == b ? taun : 0.0);
                        put(a, b, 1, fn - (a == b ? taun : 0.0) + (u[a] - uh[a]) * dtau);
                    }
                    for (int l = 0; l < 3; ++l) {
                        double qe[M][3];
                        for (int a = 0; a < M; ++a) for (int k = 0; k < 3; ++k) qe[a][k] = (a == b && k == l) ? 1.0 : 0.0;
                        double Fq[M][3];
                        visc_flux<3, double, double>(uh, qe, 0.0, P, Fq);
                        for (int a = 0; a < M; ++a) {
                            double fn = 0.0;
                            for (int k = 0; k < 3; ++k) fn += Fq[a][k] * nw[k];
                            put(a, b, 2 + l, -fn);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    if constexpr (sizeof(TJ) == sizeof(float)) {
        // A2 on the tensor cores (pairs stacked, coefficients folded into the row operand)
        contract_tc(d, tabJ, cv, cf, cb, vq, fpo, Mx, reinterpret_cast<float*>(sD), *ts, sflag);
        __syncthreads();
    } else {
        // A2: contraction into the bordered matrix, one (a, b) component pair at a time
        TJ* sR = reinterpret_cast<TJ*>(sD);  // [KC][SRP] row basis
        TJ* sT = sR + KC * SRP;              // [KC][STP] column variations times coefficients
        const TJ* dphiJ = tabJ + d.vtab + (size_t)Nq * Np;
        const TJ* phiJ = tabJ + d.vtab;
        const int nrt = (Np + 3) / 4, nct = (Nc + 3) / 4;
        const int ti = tid / nct, tc = tid - ti * nct;
        const bool act = tid < nrt * nct;
        const int K1 = 3 * Nq + sfq;         // element rows: volume (g, r) then face points
        for (int ab = 0; ab < M * M; ++ab) {
            const int a = ab / M, b = ab - a * M;
            TJ acc[4][4] = {};
            for (int k0 = 0; k0 < K1; k0 += KC) {
                const int kc = min(KC, K1 - k0);
                // operands of the chunk; four entries per thread per pass, their loads
                // issued before any store so that they are in flight together
                for (int base = tid; base < kc * SRP; base += 4 * NTH) {
                    TJ vv[4];
    #pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int idx = base + u * NTH;
                        const int kk = idx / SRP, i = idx - kk * SRP, K = k0 + kk;
                        TJ v = 0;
                        if (idx < kc * SRP && i < Np) {
                            if (K < 3 * Nq) v = dphiJ[((size_t)(K % 3) * Nq + K / 3) * Np + i];
                            else v = basis_row_t(tabJ, d, Nq + K - 3 * Nq)[i];
                        }
                        vv[u] = v;
                    }
    #pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (base + u * NTH < kc * SRP) sR[base + u * NTH] = vv[u];
                }
                for (int base = tid; base < kc * STP; base += 4 * NTH) {
                    TJ vv[4];
    #pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int idx = base + u * NTH;
                        const int kk = idx / STP, c = idx - kk * STP, K = k0 + kk;
                        TJ v = 0;
                        if (idx < kc * STP && c < Nc) {
                            if (K < 3 * Nq) {
                                const int g = K / 3, r = K - 3 * g;
                                const TJ* o = cv + (size_t)g * 300 + ((a * 3 + r) * M + b) * 4;
                                if (c < Np) v = o[0] * phiJ[(size_t)g * Np + c];
                                for (int l = 0; l < 3; ++l) v -= o[1 + l] * vq[((size_t)l * NPT + g) * NCM + c];
                            } else {
                                const int rr = K - 3 * Nq, x = Nq + rr;
                                const TJ* o = cf + (size_t)rr * 125 + (a * M + b) * 5;
                                if (c < Np) {
                                    v = o[0] * basis_row_t(tabJ, d, x)[c];
                                } else {
                                    const int f = face_of_point(d, rr);
                                    const int l = c - Np - fpo[f];
                                    if (l >= 0 && l < d.nfp[f])
                                        v = o[1] * tabJ[d.ttab[f] + (size_t)(rr - d.soff[f]) * d.nfp[f] + l];
                                }
                                for (int l = 0; l < 3; ++l) v -= o[2 + l] * vq[((size_t)l * NPT + x) * NCM + c];
                            }
                        }
                        vv[u] = v;
                    }
    #pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (base + u * NTH < kc * STP) sT[base + u * NTH] = vv[u];
                }
                __syncthreads();
                if (act) gemm_chunk(sR, sT, kc, ti, tc, acc);
                __syncthreads();
            }
            if (act)
                for (int u = 0; u < 4; ++u) {
                    const int i = 4 * ti + u;
                    if (i >= Np) continue;
                    for (int v = 0; v < 4; ++v) {
                        const int c = 4 * tc + v;
                        if (c >= Nc) continue;
                        Mx[(size_t)(a * Np + i) * LD + bcol(d, b, c)] = (double)acc[u][v];   // mass term added below
                    }
                }
            // trace rows (f', a, l'): K = the points of face f'
            for (int f2 = 0; f2 < 4; ++f2) {
                const int nfq = d.nfq[f2], nfp = d.nfp[f2];
                const TJ* mu = tabJ + d.ttab[f2];
                for (int idx = tid; idx < nfq * SRP; idx += NTH) {
                    const int kk = idx / SRP, l = idx - kk * SRP;
                    sR[idx] = l < nfp ? mu[(size_t)kk * nfp + l] : TJ(0);
                }
                for (int idx = tid; idx < nfq * STP; idx += NTH) {
                    const int kk = idx / STP, c = idx - kk * STP, rr = d.soff[f2] + kk, x = Nq + rr;
                    TJ v = 0;
                    if (c < Nc) {
                        const TJ* o = cb + (size_t)rr * 125 + (a * M + b) * 5;
                        if (c < Np) {
                            v = o[0] * basis_row_t(tabJ, d, x)[c];
                        } else {
                            const int l = c - Np - fpo[f2];
                            if (l >= 0 && l < nfp) v = o[1] * mu[(size_t)kk * nfp + l];
                        }
                        for (int l = 0; l < 3; ++l) v -= o[2 + l] * vq[((size_t)l * NPT + x) * NCM + c];
                    }
                    sT[idx] = v;
                }
                __syncthreads();
                const int nrt2 = (nfp + 3) / 4;
                const int ti2 = tid / nct, tc2 = tid - ti2 * nct;
                if (tid < nrt2 * nct) {
                    TJ acc2[4][4] = {};
                    gemm_chunk(sR, sT, nfq, ti2, tc2, acc2);
                    for (int u = 0; u < 4; ++u) {
                        const int l = 4 * ti2 + u;
                        if (l >= nfp) continue;
                        for (int v = 0; v < 4; ++v) {
                            const int c = 4 * tc2 + v;
                            if (c >= Nc) continue;
                            Mx[(size_t)(NU + d.toff[f2] + a * nfp + l) * LD + bcol(d, b, c)] = (double)acc2[u][v];
                        }
                    }
                }
                __syncthreads();
            }
        }
        __syncthreads();
    }
    // mass term (1/a_ii) M_ij on the diagonal component blocks: M = L L^T from the factor
    for (int idx = tid; idx < Np * Np; idx += NTH) {
        const int i = idx / Np, j = idx - i * Np;
        double s = 0.0;
        for (int k = 0; k <= min(i, j); ++k) s += Mm[i * NPMAX + k] * Mm[j * NPMAX + k];
        const double mv = s / A.a_ii;
        for (int a = 0; a < M; ++a) Mx[(size_t)(a * Np + i) * LD + a * Np + j] += mv;
    }
    // right-hand-side column: R_u at the lifted gradient (interior rows), the trace residual
    const int NR = NU + t;
    for (int idx = tid; idx < NR; idx += NTH) {
        double s = 0.0;
        if (idx < NU) {
            const int a = idx / Np, i = idx - a * Np;
            double mass = 0.0;
            for (int j = 0; j < Np; ++j) {
                double mij = 0.0;
                for (int k = 0; k <= min(i, j); ++k) mij += Mm[i * NPMAX + k] * Mm[j * NPMAX + k];
                mass += mij * (sU[a * Np + j] - sUs[a * Np + j]);
            }
            s = mass / A.a_ii;
            for (int g = 0; g < Nq; ++g)
                for (int r = 0; r < 3; ++r) s += dphi[((size_t)r * Nq + g) * Np + i] * rv[(g * M + a) * 3 + r];
            for (int rr = 0; rr < sfq; ++rr) s += basis_row(A, d, Nq + rr)[i] * rf[rr * M + a];
        } else {
            int f = 0, rem = idx - NU;
            while (f < 3 && rem >= M * d.nfp[f]) { rem -= M * d.nfp[f]; ++f; }
            const int a = rem / d.nfp[f], l = rem - a * d.nfp[f];
            const double* mu = A.tab + d.ttab[f];
            for (int q = 0; q < d.nfq[f]; ++q) s += mu[(size_t)q * d.nfp[f] + l] * rb[(d.soff[f] + q) * M + a];
        }
        Mx[(size_t)idx * LD + NR] = s;
    }
    __syncthreads();
    // A3 + A4: bordered elimination
    __shared__ int piv[NB];
    if constexpr (sizeof(TJ) == sizeof(double)) {
        bordered_elim<NBE>(Mx, NU, NR, NR + 1, LD, sD, sD + NRMAX * NB, piv, sflag);
    } else {
        // FP64 LU of At (interior columns only, interchanges recorded), then the
        // right-hand sides and the trace rows in FP32 (z in FP64)
        __shared__ int gpiv[M * NPMAX];
        bordered_elim<NBE>(Mx, NU, NU, NU, LD, sD, sD + NRMAX * NB, piv, sflag, gpiv);
        __syncthreads();
        trace_schur_f32<NBE>(Mx, NU, t, LD, gpiv, reinterpret_cast<float*>(W + W_VQ),
                             reinterpret_cast<float*>(W + W_CV), reinterpret_cast<float*>(sD), *ts, sflag);
    }
}

template <class TJ, int NBE>
__global__ void __launch_bounds__(NTH, 2) k_tet_linearize(KArgs A) {
    extern __shared__ double sm[];
    __shared__ TetElem d;
    __shared__ int s_idx, sflag;
    __shared__ __align__(8) uint64_t tbar[2];
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x;
    double* W = A.work + (int64_t)blockIdx.x * A.wstride;
    if (tid == 0) sflag = 0;
    TcState ts{0u, 0u, 0u};
    if constexpr (sizeof(TJ) == sizeof(float)) {
        // tensor memory and the two stage barriers of the contraction, held for the whole launch
        if ((tid >> 5) == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(&tslot)),
                         "r"(TTCOLS));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        }
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&tbar[0])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&tbar[1])), "r"(1));
            asm volatile("fence.mbarrier_init.release.cluster;");
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        ts.tmem = tslot;
        ts.bar = smem_u32(&tbar[0]);
    }
    for (;;) {
        if (tid == 0) s_idx = atomicAdd(A.next, 1);
        __syncthreads();
        const int idx = s_idx;
        if (idx >= A.E) break;
        const int64_t e = A.order[idx];
        constexpr int NW = (int)(sizeof(TetElem) / 8);
        for (int i = tid; i < NW; i += NTH)
            reinterpret_cast<int64_t*>(&d)[i] = reinterpret_cast<const int64_t*>(A.el + e)[i];
        __syncthreads();
        process_element<TJ, NBE>(A, d, W, sm, &sflag, &ts);
        __syncthreads();
    }
    if constexpr (sizeof(TJ) == sizeof(float)) {
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if ((tid >> 5) == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(ts.tmem), "r"(TTCOLS));
    }
    if (tid == 0 && sflag) atomicOr(A.status, sflag);
}

// A5: block values, column-major per block, summed over the block's element
// contributions in ascending element order; g = -(trace rows' last column)
template <class TV>
__global__ void k_tet_assemble(const TetElem* el, const double* mat, const int64_t* hoff, const int64_t* boff,
                               const int32_t* rowptr, const int32_t* col, const int32_t* cptr, const int32_t* centry,
                               int64_t F, int64_t nnzb, TV* vals) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = wid; b < nnzb; b += nw) {
        int64_t lo = 0, hi = F;                  // row face: rowptr[Fr] <= b < rowptr[Fr + 1]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (rowptr[mid] <= b) lo = mid; else hi = mid;
        }
        const int64_t Fr = lo, G = col[b];
        const int bsF = (int)(hoff[Fr + 1] - hoff[Fr]), bsG = (int)(hoff[G + 1] - hoff[G]);
        TV* out = vals + boff[b];
        for (int idx = lane; idx < bsF * bsG; idx += 32) {
            const int c = idx / bsF, r = idx - c * bsF;
            double s = 0.0;
            for (int k = cptr[b]; k < cptr[b + 1]; ++k) {
                const TetElem& d = el[centry[3 * k]];
                const int fl = centry[3 * k + 1], gl = centry[3 * k + 2];
                s += mat[d.moff + (int64_t)(d.NU + d.toff[fl] + r) * d.LD + d.NU + d.toff[gl] + c];
            }
            out[idx] = (TV)s;
        }
    }
}

__global__ void k_tet_assemble_g(const TetElem* el, const double* mat, const int64_t* hoff, const int32_t* f2e,
                                 const int32_t* f2lf, int64_t F, double* g) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t Fr = wid; Fr < F; Fr += nw) {
        int e0 = f2e[2 * Fr], e1 = f2e[2 * Fr + 1], l0 = f2lf[2 * Fr], l1 = f2lf[2 * Fr + 1];
        if (e1 >= 0 && e1 < e0) { int t = e0; e0 = e1; e1 = t; t = l0; l0 = l1; l1 = t; }
        const int bs = (int)(hoff[Fr + 1] - hoff[Fr]);
        for (int r = lane; r < bs; r += 32) {
            double s = 0.0;
            for (int side = 0; side < 2; ++side) {
                const int e = side ? e1 : e0, fl = side ? l1 : l0;
                if (e < 0) continue;
                const TetElem& d = el[e];
                s -= mat[d.moff + (int64_t)(d.NU + d.toff[fl] + r) * d.LD + d.NU + d.t];
            }
            g[hoff[Fr] + r] = s;
        }
    }
}

// y_F = sum over the row's blocks of B x_G, one CTA per block row F.  A
// row's blocks are stored back to back, so the row is one column-major
// bs_F x W matrix (W = rw[F], the summed widths of its column faces; BJ: the
// single bs_F x bs_F inverse of the diagonal block).  Thread t takes row
// t % bs_F and every S-th column from t / bs_F (S = 256 / bs_F), so one step
// of the CTA reads S bs_F consecutive values.  The matrix is streamed in
// register batches of U columns per thread, the next batch loaded before the
// current one is used, and the first batch is issued before x is gathered
// into shared memory (converted to T).  The S partial sums of a row are added
// in a fixed order.
constexpr int RMV_THREADS = 256;

template <class T, bool BJ>
__global__ void __launch_bounds__(RMV_THREADS, 4) k_tet_rowmv(const T* __restrict__ vals,
                                                           const int64_t* __restrict__ voff,
                                                           const int64_t* __restrict__ hoff,
                                                           const int32_t* __restrict__ rowptr,
                                                           const int32_t* __restrict__ col,
                                                           const int32_t* __restrict__ rw,
                                                           const double* __restrict__ x, double* __restrict__ y) {
    extern __shared__ unsigned char rmv_raw[];
    T* xs = reinterpret_cast<T*>(rmv_raw);                  // [W]
    __shared__ T part[RMV_THREADS];
    __shared__ int cst[33];
    __shared__ int64_t cg[32];
    constexpr int U = sizeof(T) == 4 ? 8 : 4;                // columns per thread and batch
    const int tid = threadIdx.x;
    const int64_t Fr = blockIdx.x;
    const int64_t h0 = hoff[Fr];
    const int bs = (int)(hoff[Fr + 1] - h0);
    const int b0 = BJ ? 0 : rowptr[Fr];
    const int nb = BJ ? 1 : rowptr[Fr + 1] - b0;
    const int W = BJ ? bs : rw[Fr];
    const T* B = vals + (BJ ? voff[Fr] : voff[b0]);
    const int S = RMV_THREADS / bs;
    const int cs = tid / bs, r = tid - cs * bs;
    const int step = S * bs;                                 // a row holds at most 75 x 525 values
    const T* p = B + cs * bs + r;
    int c = cs < S ? cs : W;                                 // threads beyond S bs_F take no columns
    int o = 0;
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = c + u * S < W ? __ldg(p + u * step) : T(0);
    if (tid < 32) {                                         // column start of each block (warp scan)
        int w = 0;
        int64_t g = 0;
        if (tid < nb) {
            const int64_t G = BJ ? Fr : col[b0 + tid];
            g = hoff[G];
            w = (int)(hoff[G + 1] - g);
        }
        int sc = w;
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, sc, off);
            if (tid >= off) sc += o;
        }
        if (tid < nb) { cst[tid + 1] = sc; cg[tid] = g; }
        if (tid == 0) cst[0] = 0;
    }
    __syncthreads();
    for (int k = tid; k < W; k += RMV_THREADS) {
        int b = 0;
        while (k >= cst[b + 1]) ++b;
        xs[k] = (T)x[cg[b] + k - cst[b]];
    }
    __syncthreads();
    T a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) a[u] = 0;
    for (; c < W; c += U * S) {
        o += U * step;
        T nv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) nv[u] = c + (U + u) * S < W ? __ldg(p + (o + u * step)) : T(0);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (c + u * S < W) a[u] = fma(v[u], xs[c + u * S], a[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = nv[u];
    }
    T acc = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) acc += a[u];
    part[tid] = acc;
    __syncthreads();
    if (tid < bs) {
        T sum = part[tid];
        for (int k = 1; k < S; ++k) sum += part[k * bs + tid];
        y[h0 + tid] = (double)sum;
    }
}

// A7: dU = -U^{-1} (z + Z dUhat_K), dQ = dq0 - G dU - H dUhat_K
// element Schur complement S^K (rows and columns NU .. NU + t of the condensed
// element matrix, local trace order) to out at skoff[e], one CTA per element
template <class TO>
__global__ void k_tet_copy_sk(const TetElem* el, const double* mat, const int64_t* skoff, int64_t E, TO* out) {
    const int64_t e = blockIdx.x;
    if (e >= E) return;
    const TetElem& d = el[e];
    const int t = d.t, NU = d.NU, LD = d.LD;
    const double* Mx = mat + d.moff;
    TO* o = out + skoff[e];
    for (int idx = threadIdx.x; idx < t * t; idx += blockDim.x) {
        const int r = idx / t, c = idx - r * t;
        o[idx] = (TO)Mx[(int64_t)(NU + r) * LD + NU + c];
    }
}

constexpr int REC_THREADS = 128;

// Interior recovery dW_K = -y_K - X_K dUhat_K (eq. local-elimination), one CTA
// per element: w = z + Z dUhat_K (one warp per interior row, lanes along the
// row), dU = -U^{-1} w by blocked back substitution, then
// dQ = Q_lift - Q + G dU + H dUhat_K per component and direction.
__global__ void __launch_bounds__(REC_THREADS) k_tet_recover(const TetElem* el, const double* mat, const double* rec,
                                                             const double* dUH, double* dQ, double* dU, int64_t E) {
    __shared__ double sH[4 * M * NFPMAX];
    __shared__ double sw[M * NPMAX];
    __shared__ double sx[M * NPMAX];
    __shared__ double sD[32 * 33];
    __shared__ double part[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t e = blockIdx.x;
    if (e >= E) return;
    const TetElem& d = el[e];
    const int Np = d.Np, NU = d.NU, t = d.t, LD = d.LD, sfp = t / M;
    const double* Mx = mat + d.moff;
    for (int i = tid; i < t; i += REC_THREADS) {
        int f = 0, r = i;
        while (f < 3 && r >= M * d.nfp[f]) { r -= M * d.nfp[f]; ++f; }
        sH[i] = dUH[d.hoff[f] + r];
    }
    __syncthreads();
    for (int i = warp; i < NU; i += REC_THREADS / 32) {
        const double* row = Mx + (int64_t)i * LD;
        double s = 0.0;
        for (int c = lane; c < t; c += 32) s = fma(row[NU + c], sH[c], s);
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) sw[i] = s + row[NU + t];
    }
    __syncthreads();
    upper_solve_blocked<REC_THREADS>(Mx, LD, NU, sw, sx, sD, part);
    for (int i = tid; i < NU; i += REC_THREADS) dU[d.uoff + i] = -sx[i];
    const double* Gk = rec + d.roff;
    const double* Hk = Gk + 3 * Np * Np;
    const double* dq0 = Hk + 3 * Np * sfp;
    for (int idx = tid; idx < 3 * NU; idx += REC_THREADS) {
        const int k = idx / NU, rem = idx - k * NU, a = rem / Np, i = rem - a * Np;
        double s = dq0[idx];
        for (int j = 0; j < Np; ++j) s += Gk[((int64_t)k * Np + i) * Np + j] * sx[a * Np + j];
        int cp = 0;
        for (int f = 0; f < 4; ++f)
            for (int l = 0; l < d.nfp[f]; ++l, ++cp)
                s -= Hk[((int64_t)k * Np + i) * sfp + cp] * sH[d.toff[f] + a * d.nfp[f] + l];
        dQ[3 * d.uoff + idx] = s;
    }
}


// FP64 stage residual of one element (eq. hdg-weak with the DIRK mass term):
// R_q, R_u into Rq / Ru (when given), the element's trace residual R_uhat^K
// into rk, the sum of squares of (R_q, R_u) into part[e]
__device__ void residual_element(const KArgs& A, const TetElem& d, int64_t e, double* W, double* sm) {
    const int tid = threadIdx.x;
    const int Np = d.Np, Nq = d.Nq, NU = d.NU, sfq = d.sfq, npt = Nq + sfq;
    const double* phi = A.tab + d.vtab;
    const double* dphi = phi + (size_t)Nq * Np;
    double* sU = sm + S_U;
    double* sUs = sm + S_US;
    double* sQ = sm + S_Q;
    double* sUH = sm + S_UH;
    double* gv = W + W_GV;
    double* gf = W + W_GF;
    double* pu = W + W_PU;
    double* pq = W + W_PQ;
    double* pd = W + W_PL;          // [NQMAX][m]: (U - U*) at the volume points
    double* ph = W + W_PH;
    double* rv = W + W_RV;
    double* rf = W + W_RF;
    double* rb = W + W_RB;
    gather_element(A, d, sm);
    load_geometry(A, d, gv, gf);
    __syncthreads();
    for (int x = tid; x < npt; x += NTH) {
        const double* br = basis_row(A, d, x);
        double u[M], q[M][3], du[M];
        for (int a = 0; a < M; ++a) { u[a] = 0.0; du[a] = 0.0; for (int k = 0; k < 3; ++k) q[a][k] = 0.0; }
        for (int j = 0; j < Np; ++j) {
            const double w = br[j];
            for (int a = 0; a < M; ++a) {
                u[a] += w * sU[a * Np + j];
                du[a] += w * (sU[a * Np + j] - sUs[a * Np + j]);
                for (int k = 0; k < 3; ++k) q[a][k] += w * sQ[(k * M + a) * Np + j];
            }
        }
        for (int a = 0; a < M; ++a) {
            pu[x * M + a] = u[a];
            for (int k = 0; k < 3; ++k) pq[(x * M + a) * 3 + k] = q[a][k];
        }
        if (x < Nq) {
            for (int a = 0; a < M; ++a) pd[x * M + a] = du[a];
            const double* g = gv + x * 10;
            const double wJ = -A.dt * g[0];
            double Fc[M][3], Fv[M][3];
            conv_flux<3, double, double>(u, A.ph, Fc);
            visc_flux<3, double, double>(u, q, 0.0, A.ph, Fv);
            for (int a = 0; a < M; ++a)
                for (int r = 0; r < 3; ++r) {
                    double s2 = 0.0;
                    for (int k = 0; k < 3; ++k) s2 += g[1 + r * 3 + k] * (Fc[a][k] - Fv[a][k]);
                    rv[(x * M + a) * 3 + r] = wJ * s2;
                }
        } else {
            const int r = x - Nq, f = face_of_point(d, r), s2 = r - d.soff[f], tag = d.tag[f];
            const double* mu = A.tab + d.ttab[f] + (size_t)s2 * d.nfp[f];
            double uh[M];
            for (int a = 0; a < M; ++a) {
                double v = 0.0;
                for (int l = 0; l < d.nfp[f]; ++l) v += mu[l] * sUH[d.toff[f] + a * d.nfp[f] + l];
                uh[a] = v;
                ph[r * M + a] = v;
            }
            const double* nw = gf + r * 3;
            const double nrm = sqrt(nw[0] * nw[0] + nw[1] * nw[1] + nw[2] * nw[2]);
            const double nh[3] = {nw[0] / nrm, nw[1] / nrm, nw[2] / nrm};
            const double tau_s = A.tau_mode ? stab_tau<3, double, double>(uh, nh, d.hinv, A.ph) : A.tau;
            double Fc[M][3], Fv[M][3];
            conv_flux<3, double, double>(uh, A.ph, Fc);
            visc_flux<3, double, double>(uh, q, 0.0, A.ph, Fv);
            for (int a = 0; a < M; ++a) {
                double fn = 0.0;
                for (int k = 0; k < 3; ++k) fn += (Fc[a][k] - Fv[a][k]) * nw[k];
                const double fh = fn + tau_s * nrm * (u[a] - uh[a]);
                rf[r * M + a] = A.dt * fh;
                rb[r * M + a] = boundary_form<M>(tag, a, fh, nrm, u, uh, tag == 1 ? A.ub[a] : 0.0, A.ew);
            }
        }
    }
    __syncthreads();
    double sq = 0.0;
    for (int idx = tid; idx < 4 * NU; idx += NTH) {
        double v = 0.0;
        if (idx < 3 * NU) {                   // R_q[k][a][i]
            const int k = idx / NU, rem = idx - k * NU, a = rem / Np, i = rem - a * Np;
            for (int g = 0; g < Nq; ++g) {
                const double* G = gv + g * 10;
                const double dk = G[1 + 0 * 3 + k] * dphi[(size_t)g * Np + i] +
                                  G[1 + 1 * 3 + k] * dphi[((size_t)Nq + g) * Np + i] +
                                  G[1 + 2 * 3 + k] * dphi[((size_t)2 * Nq + g) * Np + i];
                v += G[0] * (pq[(g * M + a) * 3 + k] * phi[(size_t)g * Np + i] + pu[g * M + a] * dk);
            }
            for (int r = 0; r < sfq; ++r) v -= gf[r * 3 + k] * ph[r * M + a] * basis_row(A, d, Nq + r)[i];
            if (A.Rq) A.Rq[3 * d.uoff + idx] = v;
        } else {                              // R_u[a][i]
            const int rem = idx - 3 * NU, a = rem / Np, i = rem - a * Np;
            double mass = 0.0;
            for (int g = 0; g < Nq; ++g) {
                mass += gv[g * 10] * phi[(size_t)g * Np + i] * pd[g * M + a];
                for (int r = 0; r < 3; ++r) v += dphi[((size_t)r * Nq + g) * Np + i] * rv[(g * M + a) * 3 + r];
            }
            v += mass / A.a_ii;
            for (int r = 0; r < sfq; ++r) v += basis_row(A, d, Nq + r)[i] * rf[r * M + a];
            if (A.Ru) A.Ru[d.uoff + rem] = v;
        }
        sq += v * v;
    }
    for (int idx = tid; idx < d.t; idx += NTH) {   // R_uhat^K[f][a][l]
        int f = 0, rem = idx;
        while (f < 3 && rem >= M * d.nfp[f]) { rem -= M * d.nfp[f]; ++f; }
        const int a = rem / d.nfp[f], l = rem - a * d.nfp[f];
        const double* mu = A.tab + d.ttab[f];
        double v = 0.0;
        for (int q = 0; q < d.nfq[f]; ++q) v += mu[(size_t)q * d.nfp[f] + l] * rb[(d.soff[f] + q) * M + a];
        A.rk[d.koff + idx] = v;
    }
    __shared__ double red[NTH / 32];
    for (int off = 16; off > 0; off >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, off);
    if ((tid & 31) == 0) red[tid >> 5] = sq;
    __syncthreads();
    if (tid == 0) {
        double s2 = 0.0;
        for (int w = 0; w < NTH / 32; ++w) s2 += red[w];
        A.part[e] = s2;
    }
}

__global__ void __launch_bounds__(NTH, 2) k_tet_residual(KArgs A) {
    extern __shared__ double sm[];
    __shared__ TetElem d;
    const int tid = threadIdx.x;
    double* W = A.work + (int64_t)blockIdx.x * A.wstride;
    for (int64_t e = blockIdx.x; e < A.E; e += gridDim.x) {
        constexpr int NW = (int)(sizeof(TetElem) / 8);
        for (int i = tid; i < NW; i += NTH)
            reinterpret_cast<int64_t*>(&d)[i] = reinterpret_cast<const int64_t*>(A.el + e)[i];
        __syncthreads();
        residual_element(A, d, e, W, sm);
        __syncthreads();
    }
}

// R_uhat of every face: the element contributions in ascending element order; squares into part
__global__ void k_tet_residual_faces(const TetElem* el, const double* rk, const int64_t* hoff, const int32_t* f2e,
                                     const int32_t* f2lf, int64_t F, double* Ruh, double* part) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t Fr = wid; Fr < F; Fr += nw) {
        int e0 = f2e[2 * Fr], e1 = f2e[2 * Fr + 1], l0 = f2lf[2 * Fr], l1 = f2lf[2 * Fr + 1];
        if (e1 >= 0 && e1 < e0) { int t = e0; e0 = e1; e1 = t; t = l0; l0 = l1; l1 = t; }
        const int bs = (int)(hoff[Fr + 1] - hoff[Fr]);
        double sq = 0.0;
        for (int r = lane; r < bs; r += 32) {
            double v = rk[el[e0].koff + el[e0].toff[l0] + r];
            if (e1 >= 0) v += rk[el[e1].koff + el[e1].toff[l1] + r];
            if (Ruh) Ruh[hoff[Fr] + r] = v;
            sq += v * v;
        }
        for (int off = 16; off > 0; off >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, off);
        if (lane == 0) part[Fr] = sq;
    }
}

// block-Jacobi set-up: explicit inverse of every diagonal block S_FF, one CTA
// per block, by in-place Gauss-Jordan elimination with partial pivoting in the
// block's own precision T (FP64 system: FP64; mixed form: FP32).  Step c swaps
// rows c and p_c, scales the pivot row and eliminates column c from every other
// row, storing column c of the inverse in place; the row interchanges are then
// undone as column interchanges in reverse order.  Row-major in shared memory
// with leading dimension bs + 1; result column-major.
template <class T>
__global__ void __launch_bounds__(256) k_tet_bj_setup(const T* vals, const int64_t* boff, const int32_t* diagb,
                                                       const int64_t* hoff, const int64_t* bjoff, T* inv,
                                                       int32_t* status) {
    extern __shared__ unsigned char bj_raw[];
    T* a = reinterpret_cast<T*>(bj_raw);                    // [bs][bs + 1]
    __shared__ T rowc[NFPMAX * M], colc[NFPMAX * M];
    __shared__ int piv[NFPMAX * M], src[NFPMAX * M];
    __shared__ int pr;
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t Fr = blockIdx.x;
    const int bs = (int)(hoff[Fr + 1] - hoff[Fr]), ld = bs + 1;
    const T* B = vals + boff[diagb[Fr]];
    for (int idx = tid; idx < bs * bs; idx += 256) {
        const int c = idx / bs, r = idx - c * bs;
        a[r * ld + c] = B[idx];
    }
    __syncthreads();
    for (int c = 0; c < bs; ++c) {
        if (tid < 32) {                                     // pivot: largest |a_rc|, r >= c, lowest r on ties
            T bv = -1;
            int bi = INT_MAX;
            for (int r = c + lane; r < bs; r += 32) {
                const T v = fabs(a[r * ld + c]);
                if (v > bv) { bv = v; bi = r; }
            }
            for (int off = 16; off > 0; off >>= 1) {
                const T ov = __shfl_down_sync(0xffffffffu, bv, off);
                const int oi = __shfl_down_sync(0xffffffffu, bi, off);
                if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
            }
            if (lane == 0) { pr = bi == INT_MAX ? c : bi; piv[c] = pr; }
        }
        __syncthreads();
        const int p = pr;
        for (int k = tid; k < bs; k += 256) {               // pivot row (after the swap); old row c into row p
            const T vc = a[c * ld + k], vp = a[p * ld + k];
            rowc[k] = vp;
            if (p != c) a[p * ld + k] = vc;
            colc[k] = k == p ? a[c * ld + c] : a[k * ld + c];   // column c after the swap (entry c unused)
        }
        __syncthreads();
        T pv = rowc[c];
        if (pv == T(0) || !isfinite(pv)) {
            if (tid == 0) atomicOr(status, pv == T(0) ? 1 : 2);
            pv = 1;
        }
        const T ip = T(1) / pv;
        for (int r = tid >> 5; r < bs; r += 8) {           // warp per row, lanes along the row
            T* ar = a + r * ld;
            if (r == c) {
                for (int k = lane; k < bs; k += 32) ar[k] = k == c ? ip : rowc[k] * ip;
            } else {
                const T f = colc[r] * ip;
                for (int k = lane; k < bs; k += 32) ar[k] = k == c ? -f : fma(-f, rowc[k], ar[k]);
            }
        }
        __syncthreads();
    }
    if (tid == 0) {                                         // column interchanges, last step first
        for (int j = 0; j < bs; ++j) src[j] = j;
        for (int c = bs - 1; c >= 0; --c) {
            const int t = src[c];
            src[c] = src[piv[c]];
            src[piv[c]] = t;
        }
    }
    __syncthreads();
    T* o = inv + bjoff[Fr];
    for (int idx = tid; idx < bs * bs; idx += 256) {
        const int j = idx / bs, r = idx - j * bs;
        o[idx] = a[r * ld + src[j]];
    }
}

namespace {

template <class T>
int tet_alloc(hdg_ctx* h, T** out, size_t count, std::string& err) {
    void* p = nullptr;
    const size_t bytes = std::max<size_t>(1, count) * sizeof(T);
    const cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? HDG_ENOMEM : HDG_ECUDA;
    }
    h->allocs.push_back(p);
    h->device_bytes += (int64_t)bytes;
    *out = static_cast<T*>(p);
    return HDG_OK;
}

template <class T>
int tet_upload(hdg_ctx* h, T** out, const std::vector<T>& v, std::string& err) {
    int rc = tet_alloc(h, out, v.size(), err);
    if (rc) return rc;
    if (!v.empty() && cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
        err = "cudaMemcpy of set-up data failed";
        return HDG_ECUDA;
    }
    return HDG_OK;
}

#define TET_CK(call)                                                                   \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            h->err = std::string(#call) + ": " + cudaGetErrorString(e_);               \
            return HDG_ECUDA;                                                          \
        }                                                                              \
    } while (0)

}  // namespace

int create_device(hdg_ctx* h, std::string& err) {
    Ctx* c = h->tet;
    int rc;
#define UP(dst, src) if ((rc = tet_upload(h, &(dst), (src), err))) return rc
    UP(c->d_el, c->el); UP(c->d_order, c->order); UP(c->d_tab, c->tab);
    UP(c->d_tabf, std::vector<float>(c->tab.begin(), c->tab.end()));
    UP(c->d_gvol, c->gvol); UP(c->d_gface, c->gface); UP(c->d_hoff, c->hoff); UP(c->d_boff, c->boff);
    UP(c->d_rowptr, c->rowptr); UP(c->d_col, c->col); UP(c->d_cptr, c->cptr); UP(c->d_centry, c->centry);
    UP(c->d_f2e, c->f2e); UP(c->d_f2lf, c->f2lf); UP(c->d_diagb, c->diagb); UP(c->d_bjoff, c->bjoff);
#undef UP
    if ((rc = tet_alloc(h, &c->d_mat, (size_t)c->n_mat, err))) return rc;
    if ((rc = tet_alloc(h, &c->d_rec, (size_t)c->n_rec, err))) return rc;
    if ((rc = tet_alloc(h, &c->d_vals, (size_t)c->n_vals, err))) return rc;
    if ((rc = tet_alloc(h, &c->d_g, (size_t)c->n_trace, err))) return rc;
    if ((rc = tet_alloc(h, &c->d_next, 1, err))) return rc;
    if ((rc = tet_alloc(h, &c->d_rk, (size_t)c->n_rk, err))) return rc;           // residual scratch: allocated
    if ((rc = tet_alloc(h, &c->d_part, (size_t)(c->E + c->F), err))) return rc;   // here so graphs can capture it
    c->bsmax = c->wmax = 0;
    std::vector<int32_t> rw(c->F);
    for (int64_t F = 0; F < c->F; ++F) {
        c->bsmax = std::max<int>(c->bsmax, (int)(c->hoff[F + 1] - c->hoff[F]));
        int w = 0;
        for (int32_t b = c->rowptr[F]; b < c->rowptr[F + 1]; ++b) w += (int)(c->hoff[c->col[b] + 1] - c->hoff[c->col[b]]);
        rw[F] = w;
        c->wmax = std::max(c->wmax, w);
        if (c->rowptr[F + 1] - c->rowptr[F] > 32) { err = "more than 32 blocks in a block row"; return HDG_EINVAL; }
    }
    if ((rc = tet_upload(h, &c->d_rw, rw, err))) return rc;
    if (c->bsmax > NFPMAX * M) { err = "trace block larger than the degree-4 face block"; return HDG_EINVAL; }
    if (cudaFuncSetAttribute(k_tet_bj_setup<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * (size_t)c->bsmax * (c->bsmax + 1))) != cudaSuccess) {
        err = "shared-memory opt-in of the block-Jacobi kernel failed";
        return HDG_ECUDA;
    }
    if ((rc = tet_alloc(h, &h->d_status, 1, err))) return rc;
    if ((rc = tet_alloc(h, &h->d_ub, M, err))) return rc;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(k_tet_linearize<double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(S_TOTAL * sizeof(double))) != cudaSuccess ||
        cudaFuncSetAttribute(k_tet_linearize<float, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(S_TOTAL * sizeof(double))) != cudaSuccess ||
        cudaFuncSetAttribute(k_tet_linearize<double, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(S_TOTAL * sizeof(double))) != cudaSuccess ||
        cudaFuncSetAttribute(k_tet_linearize<float, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(S_TOTAL * sizeof(double))) != cudaSuccess) {
        err = "shared-memory opt-in of the tetrahedral kernel failed";
        return HDG_ECUDA;
    }
    if (cudaFuncSetAttribute(k_tet_residual, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(S_TOTAL * sizeof(double))) != cudaSuccess) {
        err = "shared-memory opt-in of the tetrahedral residual kernel failed";
        return HDG_ECUDA;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tet_linearize<double, 16>, NTH,
                                                  S_TOTAL * sizeof(double));
    c->n_slots = std::max(1, nsm * std::max(1, per_sm));
    c->work_stride = W_END;
    if ((rc = tet_alloc(h, &c->d_work, (size_t)c->n_slots * W_END, err))) return rc;
    if (cudaMemset(h->d_status, 0, sizeof(int32_t)) != cudaSuccess ||
        cudaMemset(h->d_ub, 0, M * sizeof(double)) != cudaSuccess) {
        err = "cudaMemset failed";
        return HDG_ECUDA;
    }
    h->device = true;
    return HDG_OK;
}

void destroy(hdg_ctx* h) {
    delete h->tet;
    h->tet = nullptr;
}

int linearize(hdg_ctx* h, const double* U, const double* Q, const double* UH, const double* Ustar, double dt,
              double a_ii) {
    Ctx* c = h->tet;
    KArgs A;
    A.el = c->d_el; A.order = c->d_order; A.E = c->E; A.next = c->d_next;
    A.tab = c->d_tab; A.tabf = c->d_tabf; A.gvol = c->d_gvol; A.gface = c->d_gface;
    A.U = U; A.Q = Q; A.UH = UH; A.Ustar = Ustar;
    A.mat = c->d_mat; A.rec = c->d_rec; A.work = c->d_work; A.wstride = c->work_stride;
    A.ph = phys_t<double>(h->phys); A.phf = phys_t<float>(h->phys); A.dt = dt; A.a_ii = a_ii; A.tau = h->phys.tau;
    A.ub = h->d_ub; A.ew = h->e_wall; A.status = h->d_status;
    A.tau_mode = h->phys.tau_mode;
    cudaStream_t st = h->stream;
    if (h->precision != HDG_PREC_FP64 && !c->d_vals32) {
        std::string err;
        const int rc = tet_alloc(h, &c->d_vals32, (size_t)c->n_vals, err);
        if (rc) { h->err = err; return rc; }
    }
    TET_CK(cudaMemsetAsync(c->d_next, 0, sizeof(int32_t), st));
    prof_begin(h, HDG_K_ELIM);
    const size_t smem = S_TOTAL * sizeof(double);
    if (h->precision == HDG_PREC_FP64) {
        if (c->nb == 8) k_tet_linearize<double, 8><<<c->n_slots, NTH, smem, st>>>(A);
        else k_tet_linearize<double, 16><<<c->n_slots, NTH, smem, st>>>(A);
    } else {
        if (c->nb == 8) k_tet_linearize<float, 8><<<c->n_slots, NTH, smem, st>>>(A);
        else k_tet_linearize<float, 16><<<c->n_slots, NTH, smem, st>>>(A);
    }
    prof_end(h);
    TET_CK(cudaGetLastError());
    if (h->d_skout) {
        if (h->precision == HDG_PREC_FP64)
            k_tet_copy_sk<double><<<(unsigned)c->E, 256, 0, st>>>(c->d_el, c->d_mat, c->d_skoff, c->E,
                                                                  static_cast<double*>(h->d_skout));
        else
            k_tet_copy_sk<float><<<(unsigned)c->E, 256, 0, st>>>(c->d_el, c->d_mat, c->d_skoff, c->E,
                                                                 static_cast<float*>(h->d_skout));
    }
    prof_begin(h, HDG_K_ASSEMBLE);
    const unsigned gb = (unsigned)std::min<int64_t>(65535, (c->nnzb + 7) / 8);
    if (h->precision == HDG_PREC_FP64) {
        k_tet_assemble<double><<<gb, 256, 0, st>>>(c->d_el, c->d_mat, c->d_hoff, c->d_boff, c->d_rowptr, c->d_col,
                                                   c->d_cptr, c->d_centry, c->F, c->nnzb, c->d_vals);
    } else {
        k_tet_assemble<float><<<gb, 256, 0, st>>>(c->d_el, c->d_mat, c->d_hoff, c->d_boff, c->d_rowptr, c->d_col,
                                                  c->d_cptr, c->d_centry, c->F, c->nnzb, c->d_vals32);
    }
    const unsigned gf = (unsigned)std::min<int64_t>(65535, (c->F + 7) / 8);
    k_tet_assemble_g<<<gf, 256, 0, st>>>(c->d_el, c->d_mat, c->d_hoff, c->d_f2e, c->d_f2lf, c->F, c->d_g);
    prof_end(h);
    TET_CK(cudaGetLastError());
    c->have_system = true;
    c->sys_prec = h->precision == HDG_PREC_FP64 ? HDG_PREC_FP64 : HDG_PREC_MIXED;
    h->have_system = true;
    c->bj_ready = false;       // the diagonal blocks changed
    c->asm_ready = false;      // and so did the patches
    return HDG_OK;
}

int set_element_block_output(hdg_ctx* h, void* SK) {
    Ctx* c = h->tet;
    if (SK && !c->d_skoff) {
        std::vector<int64_t> off(c->E + 1, 0);
        for (int64_t e = 0; e < c->E; ++e) off[e + 1] = off[e] + (int64_t)c->el[e].t * c->el[e].t;
        std::string err;
        const int rc = tet_upload(h, &c->d_skoff, off, err);
        if (rc) { h->err = err; return rc; }
    }
    h->d_skout = SK;
    return HDG_OK;
}

int matvec(hdg_ctx* h, const double* x, double* y) {
    Ctx* c = h->tet;
    const size_t smem = (c->sys_prec == HDG_PREC_FP64 ? sizeof(double) : sizeof(float)) * (size_t)c->wmax;
    prof_begin(h, HDG_K_MATVEC);
    if (c->sys_prec == HDG_PREC_FP64)
        k_tet_rowmv<double, false><<<(unsigned)c->F, RMV_THREADS, smem, h->stream>>>(
            c->d_vals, c->d_boff, c->d_hoff, c->d_rowptr, c->d_col, c->d_rw, x, y);
    else
        k_tet_rowmv<float, false><<<(unsigned)c->F, RMV_THREADS, smem, h->stream>>>(
            c->d_vals32, c->d_boff, c->d_hoff, c->d_rowptr, c->d_col, c->d_rw, x, y);
    prof_end(h);
    TET_CK(cudaGetLastError());
    return HDG_OK;
}

int recover(hdg_ctx* h, const double* dUH, double* dQ, double* dU) {
    Ctx* c = h->tet;
    prof_begin(h, HDG_K_RECOVER);
    k_tet_recover<<<(unsigned)c->E, REC_THREADS, 0, h->stream>>>(c->d_el, c->d_mat, c->d_rec, dUH, dQ, dU, c->E);
    prof_end(h);
    TET_CK(cudaGetLastError());
    return HDG_OK;
}

namespace {
KArgs base_args(hdg_ctx* h, const double* U, const double* Q, const double* UH, const double* Ustar, double dt,
                double a_ii) {
    Ctx* c = h->tet;
    KArgs A;
    std::memset(&A, 0, sizeof(A));
    A.el = c->d_el; A.order = c->d_order; A.E = c->E; A.next = c->d_next;
    A.tab = c->d_tab; A.tabf = c->d_tabf; A.gvol = c->d_gvol; A.gface = c->d_gface;
    A.U = U; A.Q = Q; A.UH = UH; A.Ustar = Ustar;
    A.mat = c->d_mat; A.rec = c->d_rec; A.work = c->d_work; A.wstride = c->work_stride;
    A.ph = phys_t<double>(h->phys); A.phf = phys_t<float>(h->phys); A.dt = dt; A.a_ii = a_ii; A.tau = h->phys.tau;
    A.ub = h->d_ub; A.ew = h->e_wall; A.status = h->d_status;
    A.tau_mode = h->phys.tau_mode;
    return A;
}
}  // namespace

int residual(hdg_ctx* h, const double* U, const double* Q, const double* UH, const double* Ustar, double dt,
             double a_ii, double* Rq, double* Ru, double* Ruh, double* norms) {
    Ctx* c = h->tet;
    KArgs A = base_args(h, U, Q, UH, Ustar, dt, a_ii);
    A.Rq = Rq; A.Ru = Ru; A.rk = c->d_rk; A.part = c->d_part;
    cudaStream_t st = h->stream;
    prof_begin(h, HDG_K_POINT);
    k_tet_residual<<<c->n_slots, NTH, S_TOTAL * sizeof(double), st>>>(A);
    const unsigned gf = (unsigned)std::min<int64_t>(65535, (c->F + 7) / 8);
    k_tet_residual_faces<<<gf, 256, 0, st>>>(c->d_el, c->d_rk, c->d_hoff, c->d_f2e, c->d_f2lf, c->F, Ruh,
                                             c->d_part + c->E);
    k_sum_parts<<<1, 256, 0, st>>>(c->d_part, c->E, c->d_part + c->E, c->F, norms);
    prof_end(h);
    TET_CK(cudaGetLastError());
    return HDG_OK;
}

int bj_setup(hdg_ctx* h) {
    Ctx* c = h->tet;
    if (!c->have_system) { h->err = "no assembled trace system"; return HDG_EINVAL; }
    std::string err;
    int rc;
    const bool mixed = c->sys_prec != HDG_PREC_FP64;
    if (!mixed && !c->d_bj && (rc = tet_alloc(h, &c->d_bj, (size_t)c->bjoff[c->F], err))) { h->err = err; return rc; }
    if (mixed && !c->d_bj32 && (rc = tet_alloc(h, &c->d_bj32, (size_t)c->bjoff[c->F], err))) { h->err = err; return rc; }
    const unsigned g = (unsigned)c->F;
    if (!mixed)
        k_tet_bj_setup<double><<<g, 256, sizeof(double) * (size_t)c->bsmax * (c->bsmax + 1), h->stream>>>(
            c->d_vals, c->d_boff, c->d_diagb, c->d_hoff, c->d_bjoff, c->d_bj, h->d_status);
    else
        k_tet_bj_setup<float><<<g, 256, sizeof(float) * (size_t)c->bsmax * (c->bsmax + 1), h->stream>>>(
            c->d_vals32, c->d_boff, c->d_diagb, c->d_hoff, c->d_bjoff, c->d_bj32, h->d_status);
    TET_CK(cudaGetLastError());
    c->bj_ready = true;
    return HDG_OK;
}

int bj_apply(hdg_ctx* h, const double* x, double* y) {
    Ctx* c = h->tet;
    const size_t smem = (c->sys_prec == HDG_PREC_FP64 ? sizeof(double) : sizeof(float)) * (size_t)c->bsmax;
    if (c->sys_prec == HDG_PREC_FP64)
        k_tet_rowmv<double, true><<<(unsigned)c->F, RMV_THREADS, smem, h->stream>>>(
            c->d_bj, c->d_bjoff, c->d_hoff, nullptr, nullptr, nullptr, x, y);
    else
        k_tet_rowmv<float, true><<<(unsigned)c->F, RMV_THREADS, smem, h->stream>>>(
            c->d_bj32, c->d_bjoff, c->d_hoff, nullptr, nullptr, nullptr, x, y);
    TET_CK(cudaGetLastError());
    return HDG_OK;
}

}  // namespace tet
}  // namespace hdg
