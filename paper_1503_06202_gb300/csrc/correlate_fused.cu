// correlate_fused.cu -- the whole X-engine step for up to 256 inputs in one
// kernel: nibble decode (paper Sec. II-A) fused into the Hermitian correlation
// (Sec. IV-C-1, Eq. 1), with no decoded planes in HBM.
//
// At N <= 256 the separate decode dominates: it writes 2 bytes per sample to
// HBM and the correlation reads them back, so the step moves five bytes per
// (input, sample) for one byte of input.  Here a cluster of two CTAs owns a
// channel: CTA r loads, by TMA, the raw bytes of inputs r*128 .. r*128 + 127
// (128 samples per stage), its converter warps transpose and decode them into
// the K-major E4M3 planes the tensor core reads (shared memory only), and the
// leader issues cta_group::2 MMAs of M = 256, N = 256 over the pair's planes:
//     Re += A_a B_a^T + A_b B_b^T,   Im += A_b B_a^T + (-A_a) B_b^T
// with B = A (every input against every input; the epilogue keeps i <= j).
// Each CTA supplies its 128 rows of A and its half of B, so both CTAs decode
// only their own inputs.  The 256 x 256 complex accumulator fills all 512 TMEM
// columns of both CTAs; the epilogue (tcgen05.ld -> int32 triangle) follows
// each channel.  Exactness as in the two-pass path: products <= 64, partial
// sums <= 128 * 65536 = 2^23 per launch.
//
// Roles per CTA (704 threads):
//   warp 0       TMA producer: raw tiles (128 inputs x 128 samples of one channel)
//   warp 1       TMEM allocation (collective for the pair); MMA issuer (leader)
//   warps 2..17  converters: raw tile -> transposed E4M3 planes A_a (Re), A_b (Im)
//   warps 18..21 epilogue: TMEM -> packed int32 triangle
// Converter mapping: a unit is 4 inputs (4q .. 4q + 3) x 16 samples (block b);
// converter warp w (0..15) takes, for lane q, block b = (w + q) mod 8 and half
// h = ((q >> 3) & 1) ^ (w >> 3) of the block (samples 8h .. 8h + 7).  Its raw
// reads (one 32-bit word per lane, rows differing by lane) hit 32 different
// banks; its 8-byte plane writes (row 4q + m, chunk b of a 128-byte-swizzled
// tile, half h) take 16 different 8-byte slots in every half-warp.
#include "tc_ptx.cuh"
#include "nibble.cuh"
#include "xeng_internal.h"

namespace xeng {
namespace {

constexpr int kFThreads = 704;
constexpr int kFConvWarp0 = 2, kFConvWarps = 16;
constexpr int kFEpiWarp0 = 18, kFEpiWarps = 4;
constexpr int kFRaw = 128 * 128;                 // raw tile bytes
constexpr int kFPlane = 128 * 128;               // one plane tile (128 inputs x 128 samples)
constexpr int kFStageBytes = kFRaw + 2 * kFPlane;
constexpr int kFStages = 4;
constexpr uint32_t kFTmemCols = 512;
constexpr int kFBars = 3 * kFStages + 3;         // raw full, full, empty per stage; acc full, acc empty, drain
constexpr size_t kFSmem = 1024 + (size_t)kFStages * kFStageBytes + kFBars * 8 + 16;

__host__ __device__ constexpr uint32_t fused_idesc(bool neg_a)
{
    // kind::f8f6f4, D f32, A and B E4M3 K-major, N = 256, M = 256
    return (1u << 4) | (neg_a ? (1u << 13) : 0u) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}

// K-major operand, 128-byte rows, 128-byte swizzle, 8-row groups 1 KB apart.
__device__ __forceinline__ uint64_t fdesc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

struct FusedArgs {
    int64_t t0, nt;        // samples t0 .. t0 + nt - 1 of the block, nt <= 65536
    int32_t F, N, f0, nf;  // channels f0 .. f0 + nf - 1
    int32_t *acc;          // [nf][N(N+1)/2][2], channel f0 + fl at fl
    int accumulate;        // 0: store, 1: add
    int *err;
};

__global__ void __launch_bounds__(kFThreads, 1)
correlate_fused256_kernel(const __grid_constant__ CUtensorMap raw_map, const FusedArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t *sgen = smem_raw + (sbase - raw);
    const uint32_t bars = sbase + kFStages * kFStageBytes;
    auto rawf = [&](int s) { return bars + 8u * s; };
    auto full = [&](int s) { return bars + 8u * (kFStages + s); };
    auto empty = [&](int s) { return bars + 8u * (2 * kFStages + s); };
    const uint32_t accf = bars + 8u * (3 * kFStages);
    const uint32_t acce = bars + 8u * (3 * kFStages + 1);
    const uint32_t drain = bars + 8u * (3 * kFStages + 2);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem_raw + (bars + 8u * kFBars - raw));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    int *err = a.err;
    const int it_begin = (int)(blockIdx.x >> 1), it_step = (int)(gridDim.x >> 1);
    const int n_k = (int)((a.nt + 127) / 128);
    const uint16_t kBoth = 0x3;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kFStages; s++) {
            mbar_init(rawf(s), 1);
            mbar_init(full(s), 2 * kFConvWarps);  // one arrival per converter warp of both CTAs
            mbar_init(empty(s), 1);
        }
        mbar_init(accf, 1);
        mbar_init(acce, 2 * kFEpiWarps);          // one arrival per epilogue warp of both CTAs
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&raw_map) : "memory");
    }
    if (warp == 1) {  // one collective allocation for the pair: both CTAs issue it
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kFTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    cluster_sync();  // the peer's barriers and TMEM exist before anything targets them
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer (both CTAs: each its own inputs) ----------------
            int stage = 0, issued = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int it = it_begin; ok && it < a.nf; it += it_step) {
                const int f = a.f0 + it;
                for (int kc = 0; kc < n_k; kc++) {
                    if (!mbar_wait(empty(stage), phase ^ 1u, err, kDevTimeoutProducer)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(rawf(stage), kFRaw);
                    tma_load_3d(sbase + stage * kFStageBytes, &raw_map, (int)rank * 128, f, (int)(a.t0 + kc * 128),
                                rawf(stage));
                    ++issued;
                    if (++stage == kFStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                // Let the copies already issued land before the CTA can exit.
                for (int k = 1; k <= kFStages && k <= issued; k++) {
                    int s = stage - k, p = (int)phase;
                    if (s < 0) { s += kFStages; p ^= 1; }
                    (void)mbar_wait(rawf(s), (uint32_t)p, err, kDevTimeoutProducer);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            // ---------------- MMA issuer (leader CTA) ----------------
            int stage = 0;
            uint32_t phase = 0, uses = 0;
            bool ok = true;
            const uint32_t d_re = tmem, d_im = tmem + 256u;
            for (int it = it_begin; ok && it < a.nf; it += it_step) {
                if (!mbar_wait(acce, (uses & 1u) ^ 1u, err, kDevTimeoutMma)) break;
                ++uses;
                fence_after();
                for (int kc = 0; kc < n_k; kc++) {
                    if (!mbar_try_wait(full(stage), phase) && !mbar_wait(full(stage), phase, err, kDevTimeoutMma)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t pa = sbase + stage * kFStageBytes + kFRaw;  // A_a (Re)
                    const uint32_t pb = pa + kFPlane;                          // A_b (Im)
                    const uint64_t da = fdesc(pa), db = fdesc(pb);
                    #pragma unroll
                    for (int kk = 0; kk < 4; kk++) {  // +32 bytes along K = +2 in the descriptor's address field
                        const uint32_t acc = (kc != 0 || kk != 0) ? 1u : 0u;
                        mma_f8_cg2(d_re, da + 2 * kk, da + 2 * kk, fused_idesc(false), acc);
                        mma_f8_cg2(d_re, db + 2 * kk, db + 2 * kk, fused_idesc(false), 1u);
                        mma_f8_cg2(d_im, db + 2 * kk, da + 2 * kk, fused_idesc(false), acc);
                        mma_f8_cg2(d_im, da + 2 * kk, db + 2 * kk, fused_idesc(true), 1u);
                    }
                    mma_commit_cg2(empty(stage), kBoth);
                    if (++stage == kFStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit_cg2(accf, kBoth);
            }
            // Drain: every MMA issued above has finished once this completes.
            mma_commit_cg2(drain, 0x1);
            (void)mbar_wait(drain, 0u, err, kDevTimeoutMma);
        }
    } else if (warp < kFEpiWarp0) {
        // ---------------- converters ----------------
        const int cw = warp - kFConvWarp0;               // 0..15
        const int b = ((cw & 7) + lane) & 7;             // sample block of this lane
        const int h = ((lane >> 3) & 1) ^ (cw >> 3);     // which 8 samples of the block
        const int q = lane;                              // inputs 4q .. 4q + 3
        const uint32_t full_leader = mapa_rank(full(0), 0) - full(0);  // offset into the leader's window
        int stage = 0;
        uint32_t phase = 0;
        for (int it = it_begin; it < a.nf; it += it_step) {
            bool ok = true;
            for (int kc = 0; kc < n_k; kc++) {
                ok = mbar_wait_backoff(rawf(stage), phase, err, kDevTimeoutProducer, XENG_CONV_SLEEP_NS);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                const uint32_t *rt = reinterpret_cast<const uint32_t *>(sgen + stage * kFStageBytes);
                uint8_t *pre = sgen + stage * kFStageBytes + kFRaw;
                uint8_t *pim = pre + kFPlane;
                const int64_t tb = (int64_t)kc * 128 + b * 16 + h * 8;  // first sample, within the launch
                uint32_t re[4][2], im[4][2];                            // [input m][word g] (samples 4g .. 4g + 3)
                #pragma unroll
                for (int g = 0; g < 2; g++) {
                    uint32_t r[4];
                    #pragma unroll
                    for (int k = 0; k < 4; k++) {
                        const int t = b * 16 + h * 8 + g * 4 + k;
                        r[k] = (tb + g * 4 + k < a.nt) ? rt[t * 32 + q] : 0x88888888u;  // past the end: value 0
                    }
                    // transpose + decode: r[k] byte m = (sample k, input m) -> input m's codes of samples 0..3
                    decode_input4(r, 0, re[0][g], im[0][g]);
                    decode_input4(r, 1, re[1][g], im[1][g]);
                    decode_input4(r, 2, re[2][g], im[2][g]);
                    decode_input4(r, 3, re[3][g], im[3][g]);
                }
                #pragma unroll
                for (int m = 0; m < 4; m++) {
                    const int i = 4 * q + m;
                    const int off = i * 128 + ((b ^ (i & 7)) << 4) + h * 8;  // row i, chunk b, half h
                    *reinterpret_cast<uint2 *>(pre + off) = make_uint2(re[m][0], re[m][1]);
                    *reinterpret_cast<uint2 *>(pim + off) = make_uint2(im[m][0], im[m][1]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // planes visible to the MMAs
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(full(stage) + full_leader);
                if (++stage == kFStages) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            if (!ok) break;
        }
    } else {
        // ---------------- epilogue (warps 18..21 of both CTAs) ----------------
        const int q = warp & 3;                       // TMEM lane quadrant this warp may access
        const int row = q * 32 + lane;
        const uint32_t acce_leader = mapa_rank(acce, 0);
        uint32_t uses = 0;
        const int64_t N = a.N;
        const int64_t i = (int64_t)rank * 128 + row;
        const bool row_ok = i < N;
        const int64_t row_base = i * N - i * (i - 1) / 2 - i;
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16);
        for (int it = it_begin; it < a.nf; it += it_step) {
            const bool ok = mbar_wait_backoff(accf, uses & 1u, err, kDevTimeoutEpilogue, 128);
            if (!__all_sync(0xffffffffu, ok)) break;
            ++uses;
            fence_after();
            int2 *out = reinterpret_cast<int2 *>(a.acc) + (int64_t)it * (N * (N + 1) / 2);
            for (int c = 0; c < 256; c += 16) {
                uint32_t vre[16], vim[16];
                tmem_ld16(taddr + c, vre);
                tmem_ld16(taddr + 256 + c, vim);
                tmem_ld_wait();
                if (row_ok) {
                    int2 *p = out + row_base + c;  // pairs j = c + e, e = 0..15
                    const int64_t e_lo = i - c, e_hi = N - c;
                    if (a.accumulate) {
                        int2 old[16];
                        #pragma unroll
                        for (int e = 0; e < 16; e++)
                            if (e >= e_lo && e < e_hi) old[e] = p[e];
                        #pragma unroll
                        for (int e = 0; e < 16; e++)
                            if (e >= e_lo && e < e_hi)
                                p[e] = make_int2(old[e].x + __float2int_rn(__uint_as_float(vre[e])),
                                                 old[e].y + __float2int_rn(__uint_as_float(vim[e])));
                    } else {
                        #pragma unroll
                        for (int e = 0; e < 16; e++)
                            if (e >= e_lo && e < e_hi)
                                p[e] = make_int2(__float2int_rn(__uint_as_float(vre[e])),
                                                 __float2int_rn(__uint_as_float(vim[e])));
                    }
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(acce_leader);
        }
    }

    __syncwarp();
    fence_before();
    __syncthreads();
    cluster_sync();  // no copy, commit or arrival of the peer may still target this CTA
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kFTmemCols));
    }
}

}  // namespace

bool fused256_ok(const uint8_t *block, int32_t N)
{
    return N >= 1 && N <= 256 && N % 16 == 0 && (reinterpret_cast<uintptr_t>(block) & 15) == 0;
}

cudaError_t launch_correlate_fused256(const uint8_t *block, int64_t T_block, int64_t t0, int64_t nt, int32_t F,
                                      int32_t N, int32_t f0, int32_t nf, int32_t *acc, int accumulate, int *err,
                                      int num_sms, cudaStream_t s)
{
    if (nf <= 0 || nt <= 0) return cudaSuccess;
    if (!fused256_ok(block, N) || nt > kMaxChunkSamples || t0 + nt > T_block) return cudaErrorInvalidValue;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    // raw block: dims (input, channel, sample), boxes of 128 inputs x 1 channel x 128 samples;
    // inputs past N and samples past the block read as zero bytes (the converters
    // zero the samples past the launch; the inputs past N are never written)
    CUtensorMap map;
    cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)F, (cuuint64_t)T_block};
    cuuint64_t strides[2] = {(cuuint64_t)N, (cuuint64_t)N * F};
    cuuint32_t box[3] = {128, 1, 128}, estr[3] = {1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, (void *)block, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    cudaError_t e =
        cudaFuncSetAttribute(correlate_fused256_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFSmem);
    if (e != cudaSuccess) return e;
    FusedArgs a;
    a.t0 = t0;
    a.nt = nt;
    a.F = F;
    a.N = N;
    a.f0 = f0;
    a.nf = nf;
    a.acc = acc;
    a.accumulate = accumulate;
    a.err = err;
    const int clusters = nf < num_sms / 2 ? nf : num_sms / 2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * clusters, 1, 1);
    cfg.blockDim = dim3(kFThreads, 1, 1);
    cfg.dynamicSmemBytes = kFSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, correlate_fused256_kernel, map, a);
}

}  // namespace xeng
