// peaks.cu -- dense-throughput probes that give the correlator's roofline its
// denominators on the GPU at hand: tcgen05 kind::f8f6f4 (E4M3, the kind the
// tensor engine issues), tcgen05 kind::f16, the legacy warp-level INT8
// mma.sync (m16n8k32 s8 -> s32) and CUDA-core dp4a.  sm_103a has no tcgen05
// kind::i8, so the "INT8 tensor" figure available on this target is mma.sync.
//
// Each probe runs one CTA per SM issuing independent work back to back with
// operands already on chip; the host times it with CUDA events and converts
// to dense TFLOP/s (2 flops per multiply-add).
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/xeng_peaks.h"

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// M = 128 per instruction; K = 32 (8-bit) or 16 (16-bit).  kMix 0: N = 256;
// 1: N = 128; 2: the correlator's pattern -- N = 256, then two N = 128 (the
// second with A negated) into the two halves of the same 256 columns.
// kData 1: operands are E4M3 codes of pseudo-random integers in [-8, 7] (the
// correlator's operand values) instead of zeros -- the tensor core draws more
// power on live data, which matters under the board's power cap; 2: the codes
// of pseudo-random raw nibbles u / 512 (bytes 0x00..0x0F), the fused kernel's
// operands.  kMN: both operands MN-major (128-byte swizzle, 8-row groups along K
// 1 KB apart, 128-element atoms along M/N 8 KB apart), as the single-pass
// kernels lay out raw tiles; a K step of 32 rows is 4 KB.
template <bool kF8, int kMix, int kData = 0, bool kMN = false>
__global__ void __launch_bounds__(128, 1) tc_peak_kernel(int64_t iters, int *sink)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t bar;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    // E4M3 codes of -8..7
    const uint8_t codes[16] = {0xD0, 0xCE, 0xCC, 0xCA, 0xC8, 0xC4, 0xC0, 0xB8,
                               0x00, 0x38, 0x40, 0x44, 0x48, 0x4A, 0x4C, 0x4E};
    for (int k = threadIdx.x; k < 48 * 1024; k += blockDim.x) {
        uint32_t h = (uint32_t)k * 2654435761u + blockIdx.x * 40503u;
        h ^= h >> 15;
        gbase[k] = kData == 1 ? codes[h & 15] : kData == 2 ? (uint8_t)(h & 15) : (uint8_t)0;
    }
    const uint32_t bar_a = smem_u32(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    if (threadIdx.x == 0) {
        const uint32_t a = base, b = base + 16384;
        const uint32_t mn = kMN ? (1u << 15) | (1u << 16) : 0u;
        const uint32_t idesc =
            (1u << 4) | mn | ((uint32_t)((kMix == 1 ? 128 : 256) >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        const uint32_t idesc128 = (1u << 4) | ((uint32_t)(128 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        // the MN-major descriptors: leading byte offset 8 KB (the next atom along N)
        const uint64_t mn_lbo = kMN ? ((uint64_t)((8192 >> 4) - 1) << 16) : 0u;
        for (int64_t i = 0; i < iters; i++) {
            const uint32_t off = kMN ? (uint32_t)(i & 1) * 4096 : (uint32_t)(i & 3) * 32;
            if (kF8 && kMN) {
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                             ::"r"(tmem), "l"(desc_sw128(a + off) + mn_lbo), "l"(desc_sw128(b + off) + mn_lbo),
                               "r"(idesc), "r"(1));
                continue;
            }
            if (kF8) {
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                             ::"r"(tmem), "l"(desc_sw128(a + off)), "l"(desc_sw128(b + off)), "r"(idesc), "r"(1));
                if (kMix == 2) {
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                                 ::"r"(tmem), "l"(desc_sw128(a + off)), "l"(desc_sw128(b + 16384 + off)), "r"(idesc128), "r"(1));
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                                 ::"r"(tmem + 128), "l"(desc_sw128(a + off)), "l"(desc_sw128(b + off)), "r"(idesc128 | (1u << 13)), "r"(1));
                }
            } else {
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                             ::"r"(tmem), "l"(desc_sw128(a + off)), "l"(desc_sw128(b + off)), "r"(idesc), "r"(1));
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_a)
                     : "memory");
        // bounded wait (about 2 s) for the MMAs to finish
        uint64_t t0, t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        for (;;) {
            uint32_t ok;
            asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(bar_a) : "memory");
            if (ok) break;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
            if (t1 - t0 > 2000000000ull) {
                atomicExch(sink, 1);
                break;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

// 8 warps x 8 independent m16n8k32 s8 accumulators per warp.
// The single-pass kernels' MMA issue pattern with the operands standing still:
// per stage two K steps of four N = 256 MMAs (D0 += A B, D0 += A' B', D1 +=
// A' B, D1 -= A B'), MN-major operands, a commit to the stage's mbarrier, and
// before each stage a wait for the commit of the stage four back (a four-deep
// ring whose producer is instant).  kRing false: the same MMAs, one commit at the end.
template <bool kRing>
__global__ void __launch_bounds__(128, 1) tc_ring_peak_kernel(int64_t iters, int *sink)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t bars[4];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    for (int k = threadIdx.x; k < 48 * 1024; k += blockDim.x) {
        uint32_t h = (uint32_t)k * 2654435761u + blockIdx.x * 40503u;
        h ^= h >> 15;
        gbase[k] = (uint8_t)(h & 15);
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < 4; s++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[s])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    if (threadIdx.x == 0) {
        const uint32_t idesc = (1u << 4) | (1u << 15) | (1u << 16) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        const uint64_t lbo = (uint64_t)((8192 >> 4) - 1) << 16;
        const uint64_t da = desc_sw128(base) + lbo, db = desc_sw128(base + 16384) + lbo;
        bool ok = true;
        for (int64_t i = 0; ok && i < iters; i++) {
            const int s = (int)(i & 3);
            const uint32_t bar = smem_u32(&bars[s]);
            if (kRing && i >= 4) {  // bounded wait (about 2 s) for the stage four back
                const uint32_t par = (uint32_t)(((i >> 2) - 1) & 1);
                uint64_t t0, t1;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
                for (;;) {
                    uint32_t done;
                    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                                 "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(bar), "r"(par) : "memory");
                    if (done) break;
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
                    if (t1 - t0 > 2000000000ull) {
                        atomicExch(sink, 1);
                        ok = false;
                        break;
                    }
                }
                if (!ok) break;
            }
            #pragma unroll
            for (int kk = 0; kk < 2; kk++) {
                const uint64_t k4 = 256u * kk;
                const uint32_t acc = 1u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                             ::"r"(tmem), "l"(da + k4), "l"(da + k4), "r"(idesc), "r"(acc));
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                             ::"r"(tmem), "l"(db + k4), "l"(db + k4), "r"(idesc), "r"(1u));
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                             ::"r"(tmem + 256), "l"(db + k4), "l"(da + k4), "r"(idesc), "r"(acc));
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                             ::"r"(tmem + 256), "l"(da + k4), "l"(db + k4), "r"(idesc | (1u << 13)), "r"(1u));
            }
            if (kRing || i == iters - 1)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                             : "memory");
        }
        // drain: wait (bounded) for the last stages' commits
        for (int64_t i = kRing ? (iters - 4 > 0 ? iters - 4 : 0) : iters - 1; ok && i < iters; i++) {
            const uint32_t bar = smem_u32(&bars[i & 3]);
            const uint32_t par = (uint32_t)((i >> 2) & 1);
            uint64_t t0, t1;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
            for (;;) {
                uint32_t done;
                asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                             "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(bar), "r"(par) : "memory");
                if (done) break;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
                if (t1 - t0 > 2000000000ull) {
                    atomicExch(sink, 1);
                    ok = false;
                    break;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

__global__ void __launch_bounds__(256) mma_s8_peak_kernel(int64_t iters, int seed, int *sink)
{
    uint32_t a0 = seed * 0x01010101u, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, b0 = a0 ^ 5, b1 = a0 ^ 9;
    int d[8][4];
    #pragma unroll
    for (int k = 0; k < 8; k++) d[k][0] = d[k][1] = d[k][2] = d[k][3] = 0;
    for (int64_t i = 0; i < iters; i++) {
        #pragma unroll
        for (int k = 0; k < 8; k++) {
            asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                         "{%0,%1,%2,%3};"
                         : "+r"(d[k][0]), "+r"(d[k][1]), "+r"(d[k][2]), "+r"(d[k][3])
                         : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
    }
    int s = 0;
    #pragma unroll
    for (int k = 0; k < 8; k++) s += d[k][0] + d[k][1] + d[k][2] + d[k][3];
    if (s == 0x7FFFFFFF) atomicAdd(sink, s);
}

// 8 independent dp4a chains per thread.
__global__ void __launch_bounds__(256) dp4a_peak_kernel(int64_t iters, int seed, int *sink)
{
    int x = seed * 0x01010101 + threadIdx.x, y = x ^ 0x5A5A5A5A;
    int acc[8] = {0, 1, 2, 3, 4, 5, 6, 7};
    for (int64_t i = 0; i < iters; i++) {
        #pragma unroll
        for (int k = 0; k < 8; k++) acc[k] = __dp4a(x, y + k, acc[k]);
    }
    int s = 0;
    #pragma unroll
    for (int k = 0; k < 8; k++) s += acc[k];
    if (s == 0x7FFFFFFF) atomicAdd(sink, s);
}

}  // namespace

extern "C" int xeng_peak_probe(int32_t kind, int64_t iters, double *tflops, double *ms)
{
    if (!tflops || !ms || iters < 1) return -1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -5;
    int *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(int)) != cudaSuccess) return -4;
    cudaMemset(sink, 0, sizeof(int));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double flops = 0;
    const size_t smem = 48 * 1024 + 1024;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 2 && err == cudaSuccess; rep++) {  // first pass warms up
        cudaEventRecord(e0);
        switch (kind) {
        case XENG_PEAK_TC_F8F6F4:
            cudaFuncSetAttribute(tc_peak_kernel<true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            tc_peak_kernel<true, 0><<<sms, 128, smem>>>(iters, sink);
            flops = 2.0 * 128 * 256 * 32 * (double)iters * sms;
            break;
        case XENG_PEAK_TC_F8F6F4_N128:
            cudaFuncSetAttribute(tc_peak_kernel<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            tc_peak_kernel<true, 1><<<sms, 128, smem>>>(iters, sink);
            flops = 2.0 * 128 * 128 * 32 * (double)iters * sms;
            break;
        case XENG_PEAK_TC_F8F6F4_MIX:
            cudaFuncSetAttribute(tc_peak_kernel<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            tc_peak_kernel<true, 2><<<sms, 128, smem>>>(iters, sink);
            flops = 2.0 * 128 * 512 * 32 * (double)iters * sms;
            break;
        case XENG_PEAK_TC_F8F6F4_LIVE:
            cudaFuncSetAttribute(tc_peak_kernel<true, 0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            tc_peak_kernel<true, 0, 1><<<sms, 128, smem>>>(iters, sink);
            flops = 2.0 * 128 * 256 * 32 * (double)iters * sms;
            break;
        case XENG_PEAK_TC_F8F6F4_LIVE_RAW:
            cudaFuncSetAttribute(tc_peak_kernel<true, 0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            tc_peak_kernel<true, 0, 2><<<sms, 128, smem>>>(iters, sink);
            flops = 2.0 * 128 * 256 * 32 * (double)iters * sms;
            break;
        case XENG_PEAK_TC_F8F6F4_MN:
            cudaFuncSetAttribute(tc_peak_kernel<true, 0, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            tc_peak_kernel<true, 0, 2, true><<<sms, 128, smem>>>(iters, sink);
            flops = 2.0 * 128 * 256 * 32 * (double)iters * sms;
            break;
        case XENG_PEAK_TC_F8F6F4_MN_N128:
            cudaFuncSetAttribute(tc_peak_kernel<true, 1, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            tc_peak_kernel<true, 1, 2, true><<<sms, 128, smem>>>(iters, sink);
            flops = 2.0 * 128 * 128 * 32 * (double)iters * sms;
            break;
        case XENG_PEAK_TC_F8F6F4_MN_RING:
            cudaFuncSetAttribute(tc_ring_peak_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            tc_ring_peak_kernel<true><<<sms, 128, smem>>>(iters, sink);
            flops = 2.0 * 128 * 256 * 32 * 8 * (double)iters * sms;
            break;
        case XENG_PEAK_TC_F8F6F4_MN_PAIRS:
            cudaFuncSetAttribute(tc_ring_peak_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            tc_ring_peak_kernel<false><<<sms, 128, smem>>>(iters, sink);
            flops = 2.0 * 128 * 256 * 32 * 8 * (double)iters * sms;
            break;
        case XENG_PEAK_TC_F16:
            cudaFuncSetAttribute(tc_peak_kernel<false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            tc_peak_kernel<false, 0><<<sms, 128, smem>>>(iters, sink);
            flops = 2.0 * 128 * 256 * 16 * (double)iters * sms;
            break;
        case XENG_PEAK_MMA_SYNC_S8:
            mma_s8_peak_kernel<<<sms * 4, 256>>>(iters, 3, sink);
            flops = 2.0 * 16 * 8 * 32 * 8 * (double)iters * (sms * 4 * 8);
            break;
        case XENG_PEAK_DP4A:
            dp4a_peak_kernel<<<sms * 8, 256>>>(iters, 3, sink);
            flops = 2.0 * 4 * 8 * (double)iters * (sms * 8 * 256);
            break;
        default:
            err = cudaErrorInvalidValue;
        }
        cudaEventRecord(e1);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaGetLastError();
    }
    float t = 0.f;
    int flag = 0;
    if (err == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
    if (err == cudaSuccess) cudaMemcpy(&flag, sink, sizeof(int), cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess) return err == cudaErrorInvalidValue ? -1 : -5;
    if (flag) return -6;
    *ms = t;
    *tflops = flops / (t * 1e-3) / 1e12;
    return 0;
}
