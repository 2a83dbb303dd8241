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
// each channel.
//
// The planes hold the raw nibbles, not the decoded values: a byte whose low
// four bits are u (0..15) and whose high four bits are clear is the FP8 E4M3
// code of u / 512 (the subnormal binade and the first normal one share the
// spacing 2^-9), so the converters only split bytes.  With p, q the Re and Im
// nibbles and x = (p - 8) + i (q - 8), per channel and launch of n samples
//     Re V_ij = sum(p_i p_j + q_i q_j) - 8 (S_i + S_j) + 128 n,
//     Im V_ij = sum(q_i p_j - p_i q_j) + 8 (D_i - D_j),
// with S_i = P_i + Q_i, D_i = P_i - Q_i and P_i, Q_i the sums of input i's
// nibbles.  The converters form P and Q as they go; at the end of a channel
// each CTA reduces its inputs' sums and writes them into both CTAs' shared
// memory (the epilogue of a row needs the sums of every column).  The MMA sums
// are integers / 2^18 below 450 n / 2^18; with n <= 32768 per launch they stay
// below 2^24 / 2^18, where the f32 accumulation is exact.
//
// Roles per CTA (704 threads):
//   warp 0       TMA producer: raw tiles (128 inputs x 128 samples of one channel)
//   warp 1       TMEM allocation (collective for the pair); MMA issuer (leader)
//   warps 2..17  converters: raw tile -> transposed raw-nibble planes A_a (Re), A_b (Im)
//                and the inputs' nibble sums
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
constexpr int kFBars = 3 * kFStages + 7;         // raw full, full, empty per stage; acc full, acc empty, drain;
                                                 // sums full and sums empty per parity
constexpr int kFScratch = kFConvWarps * 128 * 8; // per-converter-warp partial sums (P, Q) of the CTA's 128 inputs
constexpr int kFSums = 2 * 256 * 8;              // per channel parity: (S, D) of all 256 inputs of the pair
constexpr size_t kFSmem = 1024 + (size_t)kFStages * kFStageBytes + kFScratch + kFSums + kFBars * 8 + 16;
static_assert(kFSmem <= 232448, "shared memory over the per-CTA limit");

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
    int64_t t0, nt;        // samples t0 .. t0 + nt - 1 of the block, nt <= kFusedMaxSamples
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
    const uint32_t bars = sbase + kFStages * kFStageBytes + kFScratch + kFSums;
    auto rawf = [&](int s) { return bars + 8u * s; };
    auto full = [&](int s) { return bars + 8u * (kFStages + s); };
    auto empty = [&](int s) { return bars + 8u * (2 * kFStages + s); };
    const uint32_t accf = bars + 8u * (3 * kFStages);
    const uint32_t acce = bars + 8u * (3 * kFStages + 1);
    const uint32_t drain = bars + 8u * (3 * kFStages + 2);
    auto sums_full = [&](int par) { return bars + 8u * (3 * kFStages + 3 + par); };
    auto sums_empty = [&](int par) { return bars + 8u * (3 * kFStages + 5 + par); };
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem_raw + (bars + 8u * kFBars - raw));
    // partial sums [converter warp][input] and the pair's sums [parity][input of 256], after the stage ring
    int2 *scratch = reinterpret_cast<int2 *>(sgen + kFStages * kFStageBytes);
    int2 *sums = reinterpret_cast<int2 *>(sgen + kFStages * kFStageBytes + kFScratch);
    const uint32_t sums_u32 = sbase + kFStages * kFStageBytes + kFScratch;

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
        for (int par = 0; par < 2; par++) {
            mbar_init(sums_full(par), 2 * 4);           // one arrival per reducing warp of both CTAs
            mbar_init(sums_empty(par), 2 * kFEpiWarps); // one arrival per epilogue warp of both CTAs
        }
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
        const uint32_t peer = rank ^ 1u;
        int stage = 0, local = 0;
        uint32_t phase = 0;
        for (int it = it_begin; it < a.nf; it += it_step, ++local) {
            bool ok = true;
            uint32_t sp[4] = {0, 0, 0, 0}, sq[4] = {0, 0, 0, 0};  // nibble sums of inputs 4q + m over this lane's samples
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
                        r[k] = (tb + g * 4 + k < a.nt) ? rt[t * 32 + q] : 0u;  // past the end: nibbles 0, no term
                    }
                    // transpose: r[k] byte m = (sample k, input m) -> input m's bytes of samples 0..3,
                    // then split into the Re (high) and Im (low) nibble codes
                    #pragma unroll
                    for (int m = 0; m < 4; m++) {
                        const uint32_t sel = (uint32_t)m | ((uint32_t)(4 + m) << 4);
                        const uint32_t w = __byte_perm(__byte_perm(r[0], r[1], sel), __byte_perm(r[2], r[3], sel), 0x5410);
                        re[m][g] = (w >> 4) & 0x0F0F0F0Fu;
                        im[m][g] = w & 0x0F0F0F0Fu;
                        sp[m] = __dp4a(re[m][g], 0x01010101u, sp[m]);
                        sq[m] = __dp4a(im[m][g], 0x01010101u, sq[m]);
                    }
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
            // End of the channel: every converter warp reaches both barriers below, failed or not,
            // and they OR the failures, so the warps leave together.
            if (ok) {
                int4 *sc = reinterpret_cast<int4 *>(scratch + cw * 128 + 4 * q);
                sc[0] = make_int4((int)sp[0], (int)sq[0], (int)sp[1], (int)sq[1]);
                sc[1] = make_int4((int)sp[2], (int)sq[2], (int)sp[3], (int)sq[3]);
            }
            bool fail = bar_any(1, kFConvWarps * 32, !ok);
            if (!fail && cw < 4) {
                // warps 0..3: thread k sums input k's partials and publishes (S, D) to both CTAs
                const int k = cw * 32 + lane;
                int P = 0, Q = 0;
                #pragma unroll
                for (int w = 0; w < kFConvWarps; w++) {
                    const int2 v = scratch[w * 128 + k];
                    P += v.x;
                    Q += v.y;
                }
                const int par = local & 1;
                // the buffer was last read by both CTAs' epilogues two channels ago
                ok = mbar_wait_cluster(sums_empty(par), (uint32_t)((local >> 1) & 1) ^ 1u, err, kDevTimeoutProducer);
                if (__all_sync(0xffffffffu, ok)) {
                    const uint32_t slot = sums_u32 + (uint32_t)((par * 256 + (int)rank * 128 + k) * 8);
                    sums[par * 256 + (int)rank * 128 + k] = make_int2(P + Q, P - Q);
                    st_cluster_v2(mapa_rank(slot, peer), P + Q, P - Q);
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive_cluster(mapa_rank(sums_full(par), rank));
                        mbar_arrive_cluster(mapa_rank(sums_full(par), peer));
                    }
                } else {
                    ok = false;
                }
            }
            // the scratch may be rewritten (next channel) once every reducing thread has read it
            fail = bar_any(1, kFConvWarps * 32, !ok) || fail;
            if (fail) break;
        }
    } else {
        // ---------------- epilogue (warps 18..21 of both CTAs) ----------------
        const int q = warp & 3;                       // TMEM lane quadrant this warp may access
        const int row = q * 32 + lane;
        const uint32_t acce_leader = mapa_rank(acce, 0);
        const uint32_t peer = rank ^ 1u;
        uint32_t uses = 0;
        int local = 0;
        const int64_t N = a.N;
        const int64_t i = (int64_t)rank * 128 + row;
        const bool row_ok = i < N;
        const int64_t row_base = i * N - i * (i - 1) / 2 - i;
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16);
        const int base_re = 128 * (int)a.nt;          // 64 n from each of the two products
        for (int it = it_begin; it < a.nf; it += it_step, ++local) {
            bool ok = mbar_wait_backoff(accf, uses & 1u, err, kDevTimeoutEpilogue, 128);
            const int par = local & 1;
            ok = ok && mbar_wait_cluster(sums_full(par), (uint32_t)((local >> 1) & 1), err, kDevTimeoutEpilogue);
            if (!__all_sync(0xffffffffu, ok)) break;
            ++uses;
            fence_after();
            const int2 *sm = sums + par * 256;
            const int2 si = sm[i];                    // (S_i, D_i)
            int2 *out = reinterpret_cast<int2 *>(a.acc) + (int64_t)it * (N * (N + 1) / 2);
            for (int c = 0; c < 256; c += 16) {
                uint32_t vre[16], vim[16];
                tmem_ld16(taddr + c, vre);
                tmem_ld16(taddr + 256 + c, vim);
                tmem_ld_wait();
                if (row_ok) {
                    int2 *p = out + row_base + c;  // pairs j = c + e, e = 0..15
                    const int64_t e_lo = i - c, e_hi = N - c;
                    #pragma unroll
                    for (int e = 0; e < 16; e++) {  // corrected values in place of the accumulator words
                        const int2 sj = sm[c + e];
                        // accumulators hold integer sums / 2^18: x 2^18 is exact
                        vre[e] = (uint32_t)(__float2int_rn(262144.0f * __uint_as_float(vre[e])) - 8 * (si.x + sj.x) +
                                            base_re);
                        vim[e] = (uint32_t)(__float2int_rn(262144.0f * __uint_as_float(vim[e])) + 8 * (si.y - sj.y));
                    }
                    if (a.accumulate) {
                        #pragma unroll
                        for (int e0 = 0; e0 < 16; e0 += 8) {  // in halves: fewer registers live
                            int2 old[8];
                            #pragma unroll
                            for (int e = 0; e < 8; e++)
                                if (e0 + e >= e_lo && e0 + e < e_hi) old[e] = p[e0 + e];
                            #pragma unroll
                            for (int e = 0; e < 8; e++)
                                if (e0 + e >= e_lo && e0 + e < e_hi)
                                    p[e0 + e] = make_int2(old[e].x + (int)vre[e0 + e], old[e].y + (int)vim[e0 + e]);
                        }
                    } else {
                        #pragma unroll
                        for (int e = 0; e < 16; e++)
                            if (e >= e_lo && e < e_hi) p[e] = make_int2((int)vre[e], (int)vim[e]);
                    }
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive_cluster(acce_leader);
                // this CTA's reads of the sums buffer are done: both CTAs' reducers may refill it
                mbar_arrive_cluster(mapa_rank(sums_empty(par), rank));
                mbar_arrive_cluster(mapa_rank(sums_empty(par), peer));
            }
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
    if (!fused256_ok(block, N) || nt > kFusedMaxSamples || t0 + nt > T_block) return cudaErrorInvalidValue;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    // raw block: dims (input, channel, sample), boxes of 128 inputs x 1 channel x 128 samples;
    // inputs past N and samples past the block read as zero bytes, nibbles 0 that
    // add nothing (the converters zero the samples past the launch; the inputs
    // past N are never written)
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
