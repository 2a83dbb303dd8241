// correlate_raw.cu -- the X-engine step for more than 256 inputs straight
// from the raw bytes: the nibble split (paper Sec. II-A) fused into the
// Hermitian correlation (Sec. IV-C-1, Eq. 1), with no decoded planes in HBM.
//
// A separate decode writes two plane bytes per input byte to HBM and the
// correlation reads them back, so the step moves five bytes per (input,
// sample) for one byte of input.  Here a cluster of two CTAs owns one
// upper-triangle pair (I2 <= J2) of 256-input blocks of one channel at a
// time.  CTA r loads, by TMA, the raw bytes of A inputs I2*256 + r*128 + [0,
// 128) and B inputs J2*256 + r*128 + [0, 128), 128 samples per tile, with a
// 128-byte swizzle: rows are samples, each 128 input bytes -- the canonical
// MN-major layout of an 8-bit tcgen05 operand (inputs along M or N, samples
// along K).  So its converter warps only split each byte in place: the low
// nibble stays where the TMA put it (the Im plane) and the high nibble goes
// to the same offset of the Re plane.  The leader issues cta_group::2 MMAs of
// M = 256, N = 256 over the pair's planes (both operands MN-major):
//     Re += A_re B_re^T + A_im B_im^T,   Im += A_im B_re^T + (-A_re) B_im^T
// (each CTA supplies its 128 rows of A and its half of B).  Diagonal pairs
// (I2 = J2) load and split A only and use it as B.  The 256 x 256 complex
// accumulator fills all 512 TMEM columns of both CTAs; the epilogue (tcgen05.ld
// -> int32 triangle) follows each pair.
//
// The planes hold raw nibbles: a byte whose low four bits are u (0..15) and
// whose high four bits are clear is the FP8 E4M3 code of u / 512 (the
// subnormal binade and the first normal one share the spacing 2^-9).  With p,
// q the Re and Im nibbles and x = (p - 8) + i (q - 8), over a launch of n
// samples
//     Re V_ij = sum(p_i p_j + q_i q_j) - 8 (S_i + S_j) + 128 n,
//     Im V_ij = sum(q_i p_j - p_i q_j) + 8 (D_i - D_j),
// with S = P + Q, D = P - Q and P, Q the sums of an input's nibbles, which a
// small kernel forms first (one read of the block).  The MMA sums are integers
// / 2^18 of at most 450 n; launches of at most 32,768 samples keep them below
// 2^24, exact in f32.
//
// Roles per CTA (576 threads):
//   warp 0       TMA producer: raw tiles into the Im planes of the stage ring
//   warp 1       TMEM allocation (collective for the pair); MMA issuer (leader)
//   warps 2..9   converters: each byte of the stage split into its Re and Im nibble
//   warps 10..17 epilogue: TMEM -> packed int32 triangle, two warps per TMEM lane
//                quadrant, each half of the columns
#include "tc_ptx.cuh"
#include "triangle_store.cuh"
#include "xeng_internal.h"

namespace xeng {
namespace {

constexpr int kRConvWarp0 = 2, kRConvWarps = 8;
constexpr int kREpiWarp0 = kRConvWarp0 + kRConvWarps, kREpiWarps = 8;  // two per TMEM lane quadrant
constexpr int kRThreads = 32 * (kREpiWarp0 + kREpiWarps);
// L2 prefetch distance (a build parameter): when it loads a stage, the producer
// also asks L2 for the raw tiles of the stage this many ahead in the same pair
// (0: no prefetch).  Measured on GB300 (full CHIME): none 50.8 ms, 2 / 4 / 8
// stages ahead 58.4-58.7 ms -- the extra requests cost more than they hide.
#ifndef XENG_RAW_PREFETCH
#define XENG_RAW_PREFETCH 0
#endif
// Samples per stage (a build parameter, 64 or 128): the ring holds 192 KB of
// stages of A_re, A_im, B_re, B_im, so shorter stages mean more of them in
// flight -- the TMA fills a stage's Im planes only once its MMAs have completed.
#ifndef XENG_RAW_CHUNK
#define XENG_RAW_CHUNK 128
#endif
constexpr int kRKc = XENG_RAW_CHUNK;
static_assert(kRKc == 64 || kRKc == 128, "XENG_RAW_CHUNK must be 64 or 128");
constexpr int kRTile = kRKc * 128;         // one plane tile: kRKc samples x 128 inputs
constexpr int kRStageBytes = 4 * kRTile;
constexpr int kRStages = 196608 / kRStageBytes;
constexpr int kRKSteps = kRKc / 32;        // 32-sample MMAs per stage
constexpr int kRChunks = kRTile / 16 / (32 * kRConvWarps);  // 16-byte chunks of a tile per converter thread
constexpr uint32_t kRTmemCols = 512;
// barriers: raw full, plane full, plane empty per stage; acc full, acc empty, drain
constexpr int kRBars = 3 * kRStages + 3;
constexpr int kRSums = 2 * (128 + 256) * 8;  // per item parity: (S, D) of the CTA's 128 rows and the 256 columns
static_assert(kREpiWarps * 32 >= 256, "the epilogue threads stage the 256 column sums one each");
constexpr size_t kRSmem = 1024 + (size_t)kRStages * kRStageBytes + kRSums + kRBars * 8 + 16;
static_assert(kRSmem <= 232448, "shared memory over the per-CTA limit");

// Instruction descriptor, kind::f8f6f4: D f32, A and B E4M3, both MN-major
// (bits 15, 16), N = 256, M = 256; bit 13 negates A.
__host__ __device__ constexpr uint32_t raw_idesc(bool neg_a)
{
    return (1u << 4) | (neg_a ? (1u << 13) : 0u) | (1u << 15) | (1u << 16) | ((uint32_t)(256 >> 3) << 17) |
           ((uint32_t)(256 >> 4) << 24);
}

// MN-major operand with a 128-byte swizzle: rows of 128 elements along M/N,
// 8-row groups along K 1 KB apart (stride byte offset), version 1.  A CTA's
// operand is one swizzle atom wide along M/N, so the leading byte offset (the
// step between atoms along M/N) is not used; it is set to the same 1 KB.
__device__ __forceinline__ uint64_t rdesc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(1024 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

struct RawArgs {
    int64_t t0, nt;          // samples t0 .. t0 + nt - 1 of the block, nt <= kFusedMaxSamples
    int32_t F, N, f0, nf;    // channels f0 .. f0 + nf - 1
    int32_t nt2;             // 256-input blocks
    int32_t pairs_per_ch;    // nt2 (nt2 + 1) / 2
    int32_t n_items;         // nf * pairs_per_ch
    int32_t *acc;            // [nf][N(N+1)/2][2], channel f0 + fl at fl
    const int2 *sums;        // [nf][N] (S, D) of every input over the launch's samples
    int accumulate;          // 0: store, 1: add
    int *err;
};

struct RawItem {
    int fl, I2, J2;
};

// Item `it`: channel-major, the channel's block pairs I2 <= J2 row by row.
__device__ __forceinline__ RawItem raw_item(const RawArgs &a, int it)
{
    RawItem w;
    w.fl = it / a.pairs_per_ch;
    int r = it - w.fl * a.pairs_per_ch, i = 0;
    while (r >= a.nt2 - i) {
        r -= a.nt2 - i;
        ++i;
    }
    w.I2 = i;
    w.J2 = i + r;
    return w;
}

__global__ void __launch_bounds__(kRThreads, 1)
correlate_raw_kernel(const __grid_constant__ CUtensorMap raw_map, const RawArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t *sgen = smem_raw + (sbase - raw);
    const uint32_t sums_u = sbase + kRStages * kRStageBytes;
    const uint32_t bars = sums_u + kRSums;
    int2 *srow = reinterpret_cast<int2 *>(sgen + (sums_u - sbase));  // [parity][128]
    int2 *scol = srow + 2 * 128;                                        // [parity][256]
    auto rawf = [&](int s) { return bars + 8u * s; };
    auto full = [&](int s) { return bars + 8u * (kRStages + s); };
    auto empty = [&](int s) { return bars + 8u * (2 * kRStages + s); };
    const uint32_t accf = bars + 8u * (3 * kRStages);
    const uint32_t acce = accf + 8u;
    const uint32_t drain = accf + 16u;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem_raw + (bars + 8u * kRBars - raw));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    int *err = a.err;
    const int it_begin = (int)(blockIdx.x >> 1), it_step = (int)(gridDim.x >> 1);
    const int n_k = (int)((a.nt + kRKc - 1) / kRKc);
    const uint16_t kBoth = 0x3;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kRStages; s++) {
            mbar_init(rawf(s), 1);
            mbar_init(full(s), 2 * kRConvWarps);  // one arrival per converter warp of both CTAs
            mbar_init(empty(s), 1);
        }
        mbar_init(accf, 1);
        mbar_init(acce, 2 * kREpiWarps);          // one arrival per epilogue warp of both CTAs
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&raw_map) : "memory");
    }
    if (warp == 1) {  // one collective allocation for the pair: both CTAs issue it
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kRTmemCols));
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
            for (int it = it_begin; ok && it < a.n_items; it += it_step) {
                const RawItem w = raw_item(a, it);
                const int f = a.f0 + w.fl;
                const bool diag = w.I2 == w.J2;
                const int xa = w.I2 * 256 + (int)rank * 128, xb = w.J2 * 256 + (int)rank * 128;
                for (int kc = 0; kc < n_k; kc++) {
                    // the stage's planes are free once the MMAs that read them have completed
                    if (!mbar_try_wait(empty(stage), phase ^ 1u) &&
                        !mbar_wait(empty(stage), phase ^ 1u, err, kDevTimeoutProducer)) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = sbase + stage * kRStageBytes;
                    const int z = (int)(a.t0 + (int64_t)kc * kRKc);
                    mbar_expect_tx(rawf(stage), diag ? kRTile : 2 * kRTile);
                    tma_load_3d(st + kRTile, &raw_map, xa, f, z, rawf(stage));                // -> A_im
                    if (!diag) tma_load_3d(st + 3 * kRTile, &raw_map, xb, f, z, rawf(stage));  // -> B_im
                    if (XENG_RAW_PREFETCH > 0 && kc + XENG_RAW_PREFETCH < n_k) {
                        const int zp = z + XENG_RAW_PREFETCH * kRKc;
                        tma_prefetch_3d(&raw_map, xa, f, zp);
                        if (!diag) tma_prefetch_3d(&raw_map, xb, f, zp);
                    }
                    ++issued;
                    if (++stage == kRStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                // Let the copies already issued land before the CTA can exit.
                for (int k = 1; k <= kRStages && k <= issued; k++) {
                    int s = stage - k, p = (int)phase;
                    if (s < 0) { s += kRStages; p ^= 1; }
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
            for (int it = it_begin; ok && it < a.n_items; it += it_step) {
                const RawItem w = raw_item(a, it);
                const bool diag = w.I2 == w.J2;
                if (!mbar_wait(acce, (uses & 1u) ^ 1u, err, kDevTimeoutMma)) break;
                ++uses;
                fence_after();
                for (int kc = 0; kc < n_k; kc++) {
                    if (!mbar_try_wait(full(stage), phase) && !mbar_wait(full(stage), phase, err, kDevTimeoutMma)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t st = sbase + stage * kRStageBytes;
                    const uint64_t dar = rdesc(st), dai = rdesc(st + kRTile);
                    const uint64_t dbr = diag ? dar : rdesc(st + 2 * kRTile);
                    const uint64_t dbi = diag ? dai : rdesc(st + 3 * kRTile);
                    #pragma unroll
                    for (int kk = 0; kk < kRKSteps; kk++) {  // +32 samples along K = +4 KB = +256 in the address field
                        const uint32_t acc = (kc != 0 || kk != 0) ? 1u : 0u;
                        const uint64_t k4 = 256u * kk;
                        mma_f8_cg2(d_re, dar + k4, dbr + k4, raw_idesc(false), acc);
                        mma_f8_cg2(d_re, dai + k4, dbi + k4, raw_idesc(false), 1u);
                        mma_f8_cg2(d_im, dai + k4, dbr + k4, raw_idesc(false), acc);
                        mma_f8_cg2(d_im, dar + k4, dbi + k4, raw_idesc(true), 1u);
                    }
                    mma_commit_cg2(empty(stage), kBoth);
                    if (++stage == kRStages) {
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
    } else if (warp < kREpiWarp0) {
        // ---------------- converters ----------------
        // Thread t splits 16-byte chunks t + kCT k of each tile (kCT converter
        // threads): rows (samples) (t + kCT k) / 8, physical chunk t % 8 -- a
        // quarter-warp covers one whole 128-byte row, so the accesses are
        // bank-conflict-free.  The swizzle needs no care: each byte keeps its offset.
        constexpr int kCT = 32 * kRConvWarps;
        const int t = (warp - kRConvWarp0) * 32 + lane;
        const uint32_t full_leader = mapa_rank(full(0), 0) - full(0);  // offset into the leader's window
        const int nt = (int)a.nt;  // <= kFusedMaxSamples
        int stage = 0;
        uint32_t phase = 0;
        for (int it = it_begin; it < a.n_items; it += it_step) {
            const RawItem w = raw_item(a, it);
            const bool diag = w.I2 == w.J2;
            bool ok = true;
            for (int kc = 0; kc < n_k; kc++) {
                ok = mbar_wait_backoff(rawf(stage), phase, err, kDevTimeoutProducer, XENG_CONV_SLEEP_NS);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                uint8_t *pst = sgen + stage * kRStageBytes;
                const int n_tiles = diag ? 1 : 2;
                const int rows_left = nt - kc * kRKc;  // samples of this stage inside the launch (may exceed kRKc)
                uint4 v[2][kRChunks];
                #pragma unroll
                for (int ab = 0; ab < 2; ab++)
                    #pragma unroll
                    for (int hh = 0; hh < kRChunks; hh++)
                        if (ab < n_tiles)
                            v[ab][hh] = *reinterpret_cast<const uint4 *>(pst + (2 * ab + 1) * kRTile + (t + kCT * hh) * 16);
                #pragma unroll
                for (int ab = 0; ab < 2; ab++)
                    #pragma unroll
                    for (int hh = 0; hh < kRChunks; hh++) {
                        if (ab >= n_tiles) continue;
                        const int off = (t + kCT * hh) * 16;
                        const bool in = (t + kCT * hh) / 8 < rows_left;  // rows past the launch add nothing
                        uint4 re, im;
                        re.x = in ? (v[ab][hh].x >> 4) & 0x0F0F0F0Fu : 0u;
                        re.y = in ? (v[ab][hh].y >> 4) & 0x0F0F0F0Fu : 0u;
                        re.z = in ? (v[ab][hh].z >> 4) & 0x0F0F0F0Fu : 0u;
                        re.w = in ? (v[ab][hh].w >> 4) & 0x0F0F0F0Fu : 0u;
                        im.x = in ? v[ab][hh].x & 0x0F0F0F0Fu : 0u;
                        im.y = in ? v[ab][hh].y & 0x0F0F0F0Fu : 0u;
                        im.z = in ? v[ab][hh].z & 0x0F0F0F0Fu : 0u;
                        im.w = in ? v[ab][hh].w & 0x0F0F0F0Fu : 0u;
                        *reinterpret_cast<uint4 *>(pst + 2 * ab * kRTile + off) = re;        // Re plane
                        *reinterpret_cast<uint4 *>(pst + (2 * ab + 1) * kRTile + off) = im;  // Im plane, in place
                    }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // planes visible to the MMAs
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(full(stage) + full_leader);
                if (++stage == kRStages) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            if (!ok) break;
        }
    } else {
        // ---------------- epilogue (both CTAs) ----------------
        const int q = warp & 3;                          // TMEM lane quadrant this warp may access
        const int row = q * 32 + lane;
        const int cbeg = ((warp - kREpiWarp0) >> 2) * (256 / (kREpiWarps / 4));  // this warp's columns
        const int cend = cbeg + 256 / (kREpiWarps / 4);
        const int et = (warp - kREpiWarp0) * 32 + lane;  // 0..255: sums this thread stages
        const uint32_t acce_leader = mapa_rank(acce, 0);
        uint32_t uses = 0;
        int local = 0;
        const int N = a.N;                 // <= 4096: triangle offsets within a channel fit in int
        const int n128 = 128 * (int)a.nt;  // 64 n from each of the two products
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16);
        for (int it = it_begin; it < a.n_items; it += it_step, ++local) {
            const RawItem w = raw_item(a, it);
            const int par = local & 1;
            // the item's (S, D): this CTA's rows and the pair's 256 columns; the previous
            // reader of this parity's buffers finished before the last barrier below
            {
                const int2 *sg = a.sums + (int64_t)w.fl * N;
                const int jc = w.J2 * 256 + et;
                scol[par * 256 + et] = jc < N ? sg[jc] : make_int2(0, 0);
                if (et < 128) {
                    const int ir = w.I2 * 256 + (int)rank * 128 + et;
                    srow[par * 128 + et] = ir < N ? sg[ir] : make_int2(0, 0);
                }
            }
            const bool ok = mbar_wait_backoff(accf, uses & 1u, err, kDevTimeoutEpilogue, 128);
            // the sums are staged; the barrier ORs the four warps' failures, so they leave together
            if (bar_any(1, kREpiWarps * 32, !ok)) break;
            ++uses;
            fence_after();
            const int i_warp = w.I2 * 256 + (int)rank * 128 + q * 32;  // first row of the warp
            const int i = i_warp + lane;
            const bool row_ok = i < N;
            // pair (i, j) sits at i*N - i*(i-1)/2 + (j - i) in the channel's triangle
            const int row_base = i * N - i * (i - 1) / 2 - i;
            int2 *out = reinterpret_cast<int2 *>(a.acc) + (int64_t)w.fl * ((int64_t)N * (N + 1) / 2);
            const int2 si = srow[par * 128 + row];
            const int2 *cs = scol + par * 256;
            const int jbase = w.J2 * 256;
            if (i_warp < N) {
                for (int c = cbeg; c < cend; c += 8) {
                    const int j0 = jbase + c;
                    // warp-uniform skips: chunks past the last input or below every row's diagonal
                    if (j0 >= N) break;
                    if (j0 + 7 < i_warp) continue;
                    uint32_t vre[8], vim[8];
                    tmem_ld8(taddr + c, vre);
                    tmem_ld8(taddr + 256 + c, vim);
                    tmem_ld_wait();
                    if (row_ok) {
                        #pragma unroll
                        for (int e = 0; e < 8; e++) {  // corrected values in place of the accumulator words
                            const int2 sj = cs[c + e];  // the same for every lane: a broadcast
                            // accumulators hold integer sums / 2^18: x 2^18 is exact
                            vre[e] = (uint32_t)(__float2int_rn(262144.0f * __uint_as_float(vre[e])) -
                                                8 * (si.x + sj.x) + n128);
                            vim[e] = (uint32_t)(__float2int_rn(262144.0f * __uint_as_float(vim[e])) +
                                                8 * (si.y - sj.y));
                        }
                        if (a.accumulate) put8<true>(out + row_base + j0, i - j0, N - j0, vre, vim);
                        else put8<false>(out + row_base + j0, i - j0, N - j0, vre, vim);
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
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kRTmemCols));
    }
}

// (S, D) = (P + Q, P - Q) of every input over samples t0 .. t0 + nt - 1, P and
// Q the sums of its high and low nibbles.  Thread = 16 inputs (one 16-byte
// chunk of a sample row) x one segment of samples; a warp reads 512
// consecutive bytes of a row.  The byte lanes of a word add up to 16 samples
// without carrying into each other (16 x 15 = 240), then widen.  sums must be
// zero; each thread adds its segment's totals.
__global__ void raw_sums_kernel(const uint8_t *__restrict__ block, int64_t t0, int nt, int F, int N, int f0, int nf,
                                int seg, int2 *__restrict__ sums)
{
    const int n16 = N / 16;
    const int n_seg = (nt + seg - 1) / seg;
    const int64_t total = (int64_t)n16 * nf * n_seg;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= total) return;
    const int c = (int)(tid % n16);
    const int fl = (int)((tid / n16) % nf);
    const int sgi = (int)(tid / ((int64_t)n16 * nf));
    const int s0 = sgi * seg, s1 = s0 + seg < nt ? s0 + seg : nt;
    const int64_t stride = (int64_t)F * N / 16;  // uint4 per sample row
    const uint4 *p = reinterpret_cast<const uint4 *>(block + ((t0 + s0) * F + f0 + fl) * (int64_t)N) + c;
    uint32_t P[16], Q[16];
    #pragma unroll
    for (int k = 0; k < 16; k++) P[k] = Q[k] = 0;
    for (int t = s0; t < s1; t += 16) {
        uint32_t ap[4] = {0, 0, 0, 0}, aq[4] = {0, 0, 0, 0};
        const int m = s1 - t < 16 ? s1 - t : 16;
        #pragma unroll
        for (int k = 0; k < 16; k++) {
            if (k < m) {
                const uint4 x = __ldcs(p + (int64_t)(t - s0 + k) * stride);
                ap[0] += (x.x >> 4) & 0x0F0F0F0Fu;
                ap[1] += (x.y >> 4) & 0x0F0F0F0Fu;
                ap[2] += (x.z >> 4) & 0x0F0F0F0Fu;
                ap[3] += (x.w >> 4) & 0x0F0F0F0Fu;
                aq[0] += x.x & 0x0F0F0F0Fu;
                aq[1] += x.y & 0x0F0F0F0Fu;
                aq[2] += x.z & 0x0F0F0F0Fu;
                aq[3] += x.w & 0x0F0F0F0Fu;
            }
        }
        #pragma unroll
        for (int j = 0; j < 4; j++)
            #pragma unroll
            for (int b = 0; b < 4; b++) {
                P[4 * j + b] += (ap[j] >> (8 * b)) & 0xFFu;
                Q[4 * j + b] += (aq[j] >> (8 * b)) & 0xFFu;
            }
    }
    int2 *o = sums + (int64_t)fl * N + 16 * c;
    #pragma unroll
    for (int k = 0; k < 16; k++) {
        atomicAdd(&o[k].x, (int)(P[k] + Q[k]));
        atomicAdd(&o[k].y, (int)P[k] - (int)Q[k]);
    }
}

}  // namespace

bool correlate_raw_ok(const uint8_t *block, int32_t N)
{
    return N > 256 && N <= 4096 && N % 16 == 0 && (reinterpret_cast<uintptr_t>(block) & 15) == 0;
}

cudaError_t launch_correlate_raw(const uint8_t *block, int64_t T_block, int64_t t0, int64_t nt, int32_t F, int32_t N,
                                 int32_t f0, int32_t nf, int32_t *acc, int accumulate, int2 *sums, int *err,
                                 int num_sms, cudaStream_t s)
{
    if (nf <= 0 || nt <= 0) return cudaSuccess;
    if (!correlate_raw_ok(block, N) || nt > kFusedMaxSamples || t0 < 0 || t0 + nt > T_block || T_block > 2147483647LL ||
        f0 < 0 || f0 + nf > F || num_sms < 2 || (reinterpret_cast<uintptr_t>(acc) & 7) != 0 || !sums)
        return cudaErrorInvalidValue;
    // the inputs' nibble sums first
    {
        cudaError_t e = cudaMemsetAsync(sums, 0, (size_t)nf * N * sizeof(int2), s);
        if (e != cudaSuccess) return e;
        const int64_t lanes = (int64_t)(N / 16) * nf;
        int64_t n_seg = (262144 + lanes - 1) / lanes;  // enough threads to keep HBM busy
        if (n_seg > (nt + 255) / 256) n_seg = (nt + 255) / 256;
        if (n_seg < 1) n_seg = 1;
        const int seg = (int)((nt + n_seg - 1) / n_seg);
        const int64_t threads = lanes * ((nt + seg - 1) / seg);
        raw_sums_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(block, t0, (int)nt, F, N, f0, nf, seg, sums);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int32_t nt2 = (N + 255) / 256;
    const int64_t n_items = (int64_t)nf * (nt2 * (nt2 + 1) / 2);
    if (n_items > 2147483647LL) return cudaErrorInvalidValue;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    // raw block: dims (input, channel, sample), boxes of 128 inputs x 1 channel x kRKc
    // samples with a 128-byte swizzle (the MN-major operand layout); inputs past N and
    // samples past the block read as zero bytes, nibbles 0 that add nothing (the
    // converters zero the samples past the launch; rows and columns past N are never
    // written)
    CUtensorMap map;
    cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)F, (cuuint64_t)T_block};
    cuuint64_t strides[2] = {(cuuint64_t)N, (cuuint64_t)N * F};
    cuuint32_t box[3] = {128, 1, (cuuint32_t)kRKc}, estr[3] = {1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, (void *)block, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(correlate_raw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRSmem);
    if (e != cudaSuccess) return e;
    RawArgs a;
    a.t0 = t0;
    a.nt = nt;
    a.F = F;
    a.N = N;
    a.f0 = f0;
    a.nf = nf;
    a.nt2 = nt2;
    a.pairs_per_ch = nt2 * (nt2 + 1) / 2;
    a.n_items = (int32_t)n_items;
    a.acc = acc;
    a.sums = sums;
    a.accumulate = accumulate;
    a.err = err;
    const int64_t clusters = n_items < num_sms / 2 ? n_items : num_sms / 2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * clusters), 1, 1);
    cfg.blockDim = dim3(kRThreads, 1, 1);
    cfg.dynamicSmemBytes = kRSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, correlate_raw_kernel, map, a);
}

}  // namespace xeng
