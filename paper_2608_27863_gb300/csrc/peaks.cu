// Peak-rate probes (not from the paper): one hand-written kernel per arithmetic
// pipe, each keeping that pipe busy with independent operations on data held in
// registers or shared memory, timed with CUDA events.  They measure the
// denominators of the rooflines on the running GPU:
//   0 FP64 FMA (DFMA), 8 independent chains per thread;
//   1 FP64 tensor MMA (mma.sync m8n8k4 f64), 8 independent accumulators per warp;
//   2 FP32 FMA (FFMA), 8 independent chains per thread;
//   3 TF32 on the 5th-generation tensor cores (tcgen05.mma kind::tf32, 128 x 256 x 8);
//   4 BF16 on the 5th-generation tensor cores (tcgen05.mma kind::f16 with BF16 inputs, 128 x 256 x 16);
//   5 INT8 tensor MMA (mma.sync m16n8k32 s8 -> s32; sm_103a has no tcgen05 kind::i8).
// Every wait on a tensor-core completion barrier is bounded; a wait that gives
// up latches a status bit and the probe reports HDG_ECUDA.
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/hdg.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_dfma(double* out, int iters, double a, double b) {
    double acc[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = 1e-3 * (threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) acc[i] = fma(acc[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += acc[i];
    if (s == 1234.5678) out[0] = s;   // keeps the chains live; never true for these inputs
}

__global__ void __launch_bounds__(256) k_ffma(float* out, int iters, float a, float b) {
    float acc[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = 1e-3f * (threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) acc[i] = fmaf(acc[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += acc[i];
    if (s == 1234.5678f) out[0] = s;
}

__global__ void __launch_bounds__(256) k_dmma(double* out, int iters, double a, double b) {
    double c[kChains][2];
#pragma unroll
    for (int i = 0; i < kChains; ++i) c[i][0] = c[i][1] = 1e-3 * i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(c[i][0]), "+d"(c[i][1]) : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += c[i][0] + c[i][1];
    if (s == 1234.5678) out[0] = s;
}

__global__ void __launch_bounds__(256) k_imma(int* out, int iters, int a, int b) {
    int c[kChains][4];
#pragma unroll
    for (int i = 0; i < kChains; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i)
            asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                         "{%0,%1,%2,%3};"
                         : "+r"(c[i][0]), "+r"(c[i][1]), "+r"(c[i][2]), "+r"(c[i][3])
                         : "r"(a), "r"(b), "r"(a), "r"(b), "r"(a), "r"(b));
    }
    int s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
    if (s == 123456789) out[0] = s;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major shared-memory matrix descriptor without swizzle: lbo = bytes between
// K-adjacent 8-row x 16-byte core matrices, sbo = bytes between 8-row groups.
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ bool wait_parity(uint32_t bar, uint32_t phase, int limit) {
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; ++it)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(bar), "r"(phase));
    return done != 0;
}

// One 128 x 256 accumulator in tensor memory per CTA; thread 0 issues batches of
// kBatch MMAs (K = 32 bytes of each operand row per MMA) and waits for each batch.
constexpr int kM = 128, kN = 256, kBatch = 128;

template <int KIND>   // 0: kind::tf32, 1: kind::f16 with BF16 inputs
__global__ void __launch_bounds__(128) k_tc(int batches, int32_t* status) {
    __shared__ __align__(1024) uint32_t A[kM * 8];     // 128 rows x 32 bytes
    __shared__ __align__(1024) uint32_t B[kN * 8];     // 256 rows x 32 bytes
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x;
    // operand bits: small normal values (1.0 + i / 1024 as TF32, pairs of BF16)
    for (int i = tid; i < kM * 8; i += 128) A[i] = KIND == 0 ? __float_as_uint(1.0f + (i & 1023) / 1024.f) : 0x3F803F81u;
    for (int i = tid; i < kN * 8; i += 128) B[i] = KIND == 0 ? __float_as_uint(1.0f - (i & 1023) / 2048.f) : 0x3F7F3F80u;
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_addr(&tslot)),
                     "r"(kN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(&mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tslot;
    const uint32_t fmt = KIND == 0 ? 2u : 1u;
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kN >> 3) << 17) |
                           ((uint32_t)(kM >> 4) << 24);
    const uint64_t da = desc_kmajor(smem_addr(A), 128, 256);
    const uint64_t db = desc_kmajor(smem_addr(B), 128, 256);
    const uint32_t bar = smem_addr(&mbar);
    if (tid == 0) {
        uint32_t phase = 0;
        for (int bt = 0; bt < batches; ++bt) {
            for (int i = 0; i < kBatch; ++i) {
                const uint32_t acc = (bt > 0 || i > 0) ? 1u : 0u;
                if (KIND == 0)
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                                 :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
                else
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                                 :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar));
            if (!wait_parity(bar, phase, 1 << 26)) {
                atomicOr(status, 1);
                wait_parity(bar, phase, 1 << 26);
                break;
            }
            phase ^= 1;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kN));
}

}  // namespace

extern "C" int hdg_measure_peaks(double* tflops, double* ms) {
    if (!tflops) return HDG_EINVAL;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HDG_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HDG_ECUDA;
    void* scratch = nullptr;
    if (cudaMalloc(&scratch, 256) != cudaSuccess) return HDG_ENOMEM;
    int32_t* status = static_cast<int32_t*>(scratch);
    cudaMemset(status, 0, sizeof(int32_t));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = nsm * 8;   // 8 CTAs of 256 threads per SM for the SIMT and mma.sync probes
    auto run = [&](int which, int reps) -> double {   // best time of reps launches, ms
        float best = 1e30f;
        for (int r = 0; r <= reps; ++r) {             // launch 0 warms up
            cudaEventRecord(e0);
            switch (which) {
                case 0: k_dfma<<<blocks, 256>>>((double*)scratch + 8, 8192, 0.999999, 1e-7); break;
                case 1: k_dmma<<<blocks, 256>>>((double*)scratch + 8, 2048, 0.999, 1e-7); break;
                case 2: k_ffma<<<blocks, 256>>>((float*)scratch + 16, 65536, 0.999999f, 1e-7f); break;
                case 3: k_tc<0><<<nsm * 2, 128>>>(512, status); break;
                case 4: k_tc<1><<<nsm * 2, 128>>>(512, status); break;
                case 5: k_imma<<<blocks, 256>>>((int*)scratch + 16, 2048, 0x01020304, 0x01010101); break;
            }
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (r > 0 && t < best) best = t;
        }
        return best;
    };
    const double thr = (double)blocks * 256;
    const double work[6] = {
        thr * kChains * 8192 * 2,                          // DFMA: 2 flops each
        thr / 32 * kChains * 2048 * (2.0 * 8 * 8 * 4),     // DMMA m8n8k4 per warp
        thr * kChains * 65536 * 2,                         // FFMA
        (double)nsm * 2 * 512 * kBatch * (2.0 * kM * kN * 8),    // TF32: K = 8 per MMA
        (double)nsm * 2 * 512 * kBatch * (2.0 * kM * kN * 16),   // BF16: K = 16 per MMA
        thr / 32 * kChains * 2048 * (2.0 * 16 * 8 * 32),   // IMMA m16n8k32 per warp
    };
    int rc = HDG_OK;
    for (int w = 0; w < 6; ++w) {
        const double t = run(w, 3);
        tflops[w] = work[w] / (t * 1e-3) / 1e12;
        if (ms) ms[w] = t;
    }
    int32_t st = 0;
    if (cudaMemcpy(&st, status, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess || st != 0) rc = HDG_ECUDA;
    if (cudaGetLastError() != cudaSuccess) rc = HDG_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(scratch);
    return rc;
}
