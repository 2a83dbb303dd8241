// correlate_tc.cu -- Hermitian correlation on the 5th-generation tensor cores.
//
// Computes, for every channel of a group and every upper-triangle tile pair
// (I <= J) of 128 x 128 inputs, the visibility block (paper Sec. IV-C-1, Eq. 1)
//     V_ij = sum_t x_i(t) conj(x_j(t)),   i in tile I, j in tile J,
// as a real GEMM on decoded planes a = Re x, b = Im x (K = samples), with the
// A operand from tile J (TMEM lanes are inputs j) and B from tile I (columns
// are inputs i):
//     D[:, 0:128]   = A_a B_a^T + A_b B_b^T          = Re V
//     D[:, 128:256] = A_a B_b^T - A_b B_a^T          = Im V
// issued per 32-sample K step as three tcgen05.mma (kind::f8f6f4, E4M3 x E4M3
// -> f32 in TMEM):
//     D[:, 0:256]  += A_a x [B_a ; B_b]^T      (N = 256, B_b follows B_a in smem)
//     D[:, 0:128]  += A_b x B_b^T              (N = 128)
//     D[:, 128:256]+= (-A_b) x B_a^T           (N = 128, A negated by the
//                                               instruction descriptor)
// Every product is an integer of magnitude <= 64 and every partial sum an
// integer of magnitude <= 128 * 65536 = 2^23, so the f32 accumulation is exact
// provided the tensor core adds without dropping bits below 2^24; the tests
// check this against the integer oracle on adversarial inputs.
//
// Structure: persistent CTAs (one per SM), static round-robin over tiles,
// channel-major so one channel's operands stay in L2 while its tiles run.
//   warp 0      TMA producer: 128x128-byte SWIZZLE_128B boxes of the planes
//   warp 1      TMEM allocator and single-thread MMA issuer
//   warps 2..5  epilogue: tcgen05.ld -> int32 -> packed triangle in HBM; per
//               column i a warp's 32 lanes write 32 consecutive pairs of the
//               triangle's row i (one 256-byte run, 8-byte aligned whatever
//               the row's start)
// Smem ring of 3 stages x 64 KB (A_a, A_b, B_a, B_b of a 128-sample chunk;
// diagonal tiles load only A and reuse it as B).  Two 256-column TMEM
// accumulators let the epilogue of one tile overlap the MMAs of the next.
// Every wait is bounded: on time-out the thread records a status in the
// error word, the others see it and leave their loops, the MMA thread drains
// its tensor-core work and TMEM is freed before the CTA exits.
#include <cstring>
#include <vector>

#include "tc_ptx.cuh"
#include "xeng_internal.h"

namespace xeng {
namespace {

// Samples per pipeline stage (the K extent of one TMA box): 128 with a
// 128-byte swizzle, or 64 with a 64-byte swizzle (twice the stages of half the
// size in the same shared memory).  A build parameter.
#ifndef XENG_TC_CHUNK
#define XENG_TC_CHUNK 128
#endif
constexpr int kKc = XENG_TC_CHUNK;
static_assert(kKc == 128 || kKc == 64, "XENG_TC_CHUNK must be 128 or 64");
constexpr int kPlaneTile = kTile * kKc;       // 128 rows x kKc bytes
constexpr int kStageBytes = 4 * kPlaneTile;   // A_a, A_b, B_a, B_b
constexpr int kStages = (3 * 4 * kTile * 128) / kStageBytes;  // 192 KB of stages
constexpr int kKSteps = kKc / 32;             // 32-sample MMAs per stage
constexpr int kChunksPer128 = 128 / kKc;

constexpr int kThreads = 192;
constexpr uint32_t kTmemCols = 512;
constexpr int kNumBars = 2 * kStages + 5;     // full, empty, acc_full x2, acc_empty x2, drain
constexpr size_t kSmemBytes = 1024 + (size_t)kStages * kStageBytes + kNumBars * 8 + 16;

// Instruction descriptor, kind::f8f6f4: D f32 (bits 4-5 = 1), A and B E4M3
// (formats 0), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28,
// bit 13 negates A.
__host__ __device__ constexpr uint32_t make_idesc(int n, bool neg_a)
{
    return (1u << 4) | (neg_a ? (1u << 13) : 0u) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
constexpr uint32_t kIdescN256 = make_idesc(256, false);
constexpr uint32_t kIdescN128 = make_idesc(128, false);
constexpr uint32_t kIdescN128Neg = make_idesc(128, true);

// Shared-memory matrix descriptor: K-major, rows of kKc bytes swizzled over
// kKc bytes (layout 2 = 128-byte, 4 = 64-byte swizzle), 8-row groups 8 * kKc
// bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)((8 * kKc) >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)(kKc == 128 ? 2 : 4) << 61);
}

// Upper-triangle tile pair number r (row-major over I <= J) of an nt x nt grid.
__device__ __forceinline__ void tile_pair(int r, int nt, int &I, int &J)
{
    int i = 0;
    while (r >= nt - i) {
        r -= nt - i;
        ++i;
    }
    I = i;
    J = i + r;
}

struct Sched {
    int nt, tiles_per_ch, n_tiles;
    __device__ __forceinline__ void decode(int tile, int &fl, int &I, int &J) const
    {
        fl = tile / tiles_per_ch;
        tile_pair(tile - fl * tiles_per_ch, nt, I, J);
    }
};

enum EpiMode : int { kStore = 0, kAdd = 1, kAtomicAdd = 2 };

// One unit of work as every role of the CTA sees it.
struct Work {
    const CUtensorMap *map;
    int32_t *out;    // channel 0 of the job's [F][B][2] triangle
    int n_pad, N;
    int fl, I, J;
    int kc0, kc1;    // 128-sample chunks [kc0, kc1)
    int mode;
    // raw-nibble planes: (S, D) of the channel's inputs (null: decoded planes),
    // 128 x samples of the integration, and whether this item adds the offset
    // terms (items split along time add them once, in the first part)
    const int2 *sums;
    int n128;
    bool offset;
};



template <bool kListed>
__device__ __forceinline__ Work fetch_work(int it, const CUtensorMap *tmap, const TcArgs &a, const Sched &sc, int n_k,
                                           const ListArgs &L)
{
    Work w;
    if (kListed) {
        const WorkItem wi = L.items[it];
        const JobDesc &jd = L.jobs[wi.job];
        w.map = &L.maps[wi.job];
        w.out = jd.out;
        w.n_pad = jd.n_pad;
        w.N = jd.N;
        w.fl = wi.fl;
        w.I = wi.I;
        w.J = wi.J;
        w.kc0 = wi.kc0 * kChunksPer128;
        w.kc1 = wi.kc1 * kChunksPer128;
        w.mode = jd.mode;
        w.sums = jd.sums ? jd.sums + (int64_t)wi.fl * jd.n_pad : nullptr;
        w.n128 = 128 * jd.n_samples;
        w.offset = wi.kc0 == 0;
    } else {
        w.map = tmap;
        w.out = a.acc;
        w.n_pad = a.n_pad;
        w.N = a.N;
        sc.decode(it, w.fl, w.I, w.J);
        w.kc0 = 0;
        w.kc1 = n_k;
        w.mode = a.accumulate ? kAdd : kStore;
        w.sums = a.sums ? a.sums + (int64_t)w.fl * a.n_pad : nullptr;
        w.n128 = 128 * (int)a.n_samples;
        w.offset = true;
    }
    return w;
}

// Persistent CTA (one per SM).  Single-instance launches walk the tiles of
// `sc` round-robin; listed launches (batches) walk items
// [cta_begin[b], cta_begin[b + 1]) of a host-planned work list.
// kRaw: the planes hold raw nibbles p (Re), q (Im) as E4M3 codes of u / 512, so
// the accumulators hold sum(p p' + q q') / 2^18 and sum(p q' - q p') / 2^18;
// with x = (p - 8) + i (q - 8) over n samples and the inputs' (S, D) =
// (P + Q, P - Q) nibble sums in a.sums,
//     Re V = sum(p p' + q q') - 8 (S_i + S_j) + 128 n,
//     -Im V = sum(p q' - q p') - 8 (D_i - D_j),
// formed right after the TMEM loads (launches of at most 32,768 samples keep
// the sums below 2^24, exact in the f32 accumulators).  Listed launches take
// raw-nibble or decoded planes per job (JobDesc::sums).
// The operands draw less power than codes of -8..7 (measured: the dense rate
// on random raw-nibble codes equals the rate on zeros, 10% above -8..7).
template <bool kListed, bool kRaw = false>
__global__ void __launch_bounds__(kThreads, 1)
correlate_tc_kernel(const __grid_constant__ CUtensorMap tmap, const TcArgs a, const Sched sc, const int n_k,
                    const ListArgs L)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    const uint32_t bars = sbase + kStages * kStageBytes;
    auto full_bar = [&](int s) { return bars + 8u * s; };
    auto empty_bar = [&](int s) { return bars + 8u * (kStages + s); };
    auto accf_bar = [&](int b) { return bars + 8u * (2 * kStages + b); };
    auto acce_bar = [&](int b) { return bars + 8u * (2 * kStages + 2 + b); };
    const uint32_t drain_bar = bars + 8u * (2 * kStages + 4);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem_raw + (bars + 8u * kNumBars - raw));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *err = kListed ? L.err : a.err;
    const bool strided = !kListed || L.cta_begin == nullptr;
    int it_begin = strided ? (int)blockIdx.x : L.cta_begin[blockIdx.x];
    int it_end = !kListed ? sc.n_tiles : (strided ? (int)L.n_items : L.cta_begin[blockIdx.x + 1]);
    int it_step = strided ? (int)gridDim.x : 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(accf_bar(b), 1);
            mbar_init(acce_bar(b), 128);
        }
        mbar_init(drain_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!kListed) asm volatile("prefetch.tensormap [%0];" ::"l"(&tmap) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int stage = 0;
            uint32_t phase = 0;
            int issued = 0;
            bool ok = true;
            for (int it = it_begin; ok && it < it_end; it += it_step) {
                const Work w = fetch_work<kListed>(it, &tmap, a, sc, n_k, L);
                const bool diag = (w.I == w.J);
                const int rowA = w.fl * 2 * w.n_pad + w.J * kTile;  // A: tile J (TMEM lanes = inputs j)
                const int rowB = w.fl * 2 * w.n_pad + w.I * kTile;  // B: tile I (columns = inputs i)
                for (int kc = w.kc0; kc < w.kc1; kc++) {
                    if (!mbar_try_wait(empty_bar(stage), phase ^ 1u) &&
                        !mbar_wait(empty_bar(stage), phase ^ 1u, err, kDevTimeoutProducer)) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = sbase + stage * kStageBytes;
                    mbar_expect_tx(full_bar(stage), diag ? 2 * kPlaneTile : 4 * kPlaneTile);
                    tma_load_2d(st, w.map, kc * kKc, rowA, full_bar(stage));
                    tma_load_2d(st + kPlaneTile, w.map, kc * kKc, rowA + w.n_pad, full_bar(stage));
                    if (!diag) {
                        tma_load_2d(st + 2 * kPlaneTile, w.map, kc * kKc, rowB, full_bar(stage));
                        tma_load_2d(st + 3 * kPlaneTile, w.map, kc * kKc, rowB + w.n_pad, full_bar(stage));
                    }
                    ++issued;
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                // Let the copies already issued land before the CTA can exit.
                for (int k = 1; k <= kStages && k <= issued; k++) {
                    int s = stage - k, p = (int)phase;
                    if (s < 0) { s += kStages; p ^= 1; }
                    (void)mbar_wait(full_bar(s), (uint32_t)p, err, kDevTimeoutProducer);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            int stage = 0;
            uint32_t phase = 0;
            uint32_t uses[2] = {0, 0};
            bool ok = true;
            int local = 0;
            for (int it = it_begin; ok && it < it_end; it += it_step, ++local) {
                const Work w = fetch_work<kListed>(it, &tmap, a, sc, n_k, L);
                const bool diag = (w.I == w.J);
                const int ab = local & 1;
                if (!mbar_wait(acce_bar(ab), (uses[ab] & 1u) ^ 1u, err, kDevTimeoutMma)) break;
                ++uses[ab];
                fence_after();
                const uint32_t d = tmem + (uint32_t)ab * 256u;
                for (int kc = w.kc0; kc < w.kc1; kc++) {
                    // inline probe first: the out-of-line bounded wait only when the stage is not there yet
                    if (!mbar_try_wait(full_bar(stage), phase) &&
                        !mbar_wait(full_bar(stage), phase, err, kDevTimeoutMma)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t st = sbase + stage * kStageBytes;
                    const uint32_t a_re = st, a_im = st + kPlaneTile;
                    const uint32_t b_re = diag ? a_re : st + 2 * kPlaneTile;
                    const uint32_t b_im = b_re + kPlaneTile;
                    // descriptors built once per stage; +32 bytes along K is +2 in their address field
                    const uint64_t dar = sw128_desc(a_re), dai = sw128_desc(a_im);
                    const uint64_t dbr = sw128_desc(b_re), dbi = sw128_desc(b_im);
                    const uint32_t acc0 = kc != w.kc0 ? 1u : 0u;
                    #pragma unroll
                    for (int kk = 0; kk < kKSteps; kk++) {
                        const uint64_t k2 = 2u * kk;
                        mma_f8(d, dar + k2, dbr + k2, kIdescN256, kk != 0 ? 1u : acc0);
                        mma_f8(d, dai + k2, dbi + k2, kIdescN128, 1u);
                        mma_f8(d + 128u, dai + k2, dbr + k2, kIdescN128Neg, 1u);
                    }
                    mma_commit(empty_bar(stage));
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit(accf_bar(ab));
            }
            // Drain: every MMA issued above has finished once this completes.
            mma_commit(drain_bar);
            (void)mbar_wait(drain_bar, 0u, err, kDevTimeoutMma);
        }
    } else {
        // ---------------- epilogue (warps 2..5) ----------------
        const int q = warp & 3;  // TMEM lane quadrant this warp may access
        const int row = q * 32 + lane;
        uint32_t uses[2] = {0, 0};
        int local = 0;
        for (int it = it_begin; it < it_end; it += it_step, ++local) {
            const Work w = fetch_work<kListed>(it, &tmap, a, sc, n_k, L);
            const int ab = local & 1;
            const bool ok = mbar_wait(accf_bar(ab), uses[ab] & 1u, err, kDevTimeoutEpilogue);
            if (!__all_sync(0xffffffffu, ok)) break;  // keep the warp converged for tcgen05.ld
            ++uses[ab];
            fence_after();
            const int N = w.N;  // <= 4096: offsets within a channel's triangle fit in int
            const int j_warp = w.J * kTile + q * 32;  // the warp's first input j
            const int j = j_warp + lane;
            const bool lane_ok = j < N;
            int2 *out = reinterpret_cast<int2 *>(w.out + (int64_t)w.fl * N * (N + 1));
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)ab * 256u;
            const int ibase = w.I * kTile;
            const bool raw = kRaw || (kListed && w.sums != nullptr);  // uniform over the item
            const int2 *sums = w.sums;                                // (S, D) per input row
            int2 sj = make_int2(0, 0);
            if (raw && w.offset) sj = sums[j];  // j < n_pad
            const int n128 = raw && w.offset ? w.n128 : 0;
            // the triangle is written once and not read again here: streaming
            // stores keep it from evicting the operand planes other tiles
            // still read from L2
            #pragma unroll 1
            for (int c = 0; c < kTile; c += 16) {
                const int i0 = ibase + c;
                // warp-uniform: columns past the last input or past every lane's diagonal
                if (i0 >= N || i0 > j_warp + 31) break;
                uint32_t re[16], im[16];
                tmem_ld16(taddr + c, re);
                tmem_ld16(taddr + 128 + c, im);
                tmem_ld_wait();
                int vr[16], vi[16];
                #pragma unroll
                for (int e = 0; e < 16; e++) {
                    if (raw) {
                        // accumulators hold integer sums / 2^18: x 2^18 is exact
                        const int2 si = w.offset ? sums[i0 + e] : make_int2(0, 0);  // a broadcast; i < n_pad
                        vr[e] = __float2int_rn(262144.0f * __uint_as_float(re[e])) - 8 * (si.x + sj.x) + n128;
                        vi[e] = __float2int_rn(262144.0f * __uint_as_float(im[e])) + 8 * (si.y - sj.y);
                    } else {
                        vr[e] = __float2int_rn(__uint_as_float(re[e]));
                        vi[e] = __float2int_rn(__uint_as_float(im[e]));
                    }
                }
                // pair (i, j) sits at i*N - i*(i-1)/2 + (j - i) in the channel's triangle;
                // row i + 1 starts N - i - 1 pairs after row i
                const int off0 = i0 * N - i0 * (i0 - 1) / 2 - i0 + j;
                if (w.mode == kStore) {
                    int off = off0;
                    #pragma unroll
                    for (int e = 0; e < 16; e++) {
                        if (lane_ok && i0 + e <= j && i0 + e < N) __stcs(out + off, make_int2(vr[e], vi[e]));
                        off += N - (i0 + e) - 1;
                    }
                } else if (w.mode == kAdd) {
                    // all 16 loads issued before any store, so they overlap in flight
                    int2 old[16];
                    int off = off0;
                    #pragma unroll
                    for (int e = 0; e < 16; e++) {
                        if (lane_ok && i0 + e <= j && i0 + e < N) old[e] = __ldcs(out + off);
                        off += N - (i0 + e) - 1;
                    }
                    off = off0;
                    #pragma unroll
                    for (int e = 0; e < 16; e++) {
                        if (lane_ok && i0 + e <= j && i0 + e < N)
                            __stcs(out + off, make_int2(old[e].x + vr[e], old[e].y + vi[e]));
                        off += N - (i0 + e) - 1;
                    }
                } else {
                    int off = off0;
                    #pragma unroll
                    for (int e = 0; e < 16; e++) {
                        if (lane_ok && i0 + e <= j && i0 + e < N) {
                            atomicAdd(&out[off].x, vr[e]);
                            atomicAdd(&out[off].y, vi[e]);
                        }
                        off += N - (i0 + e) - 1;
                    }
                }
            }
            fence_before();
            mbar_arrive(acce_bar(ab));
        }
    }

    __syncwarp();
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// Self-test of the bounded wait: thread 0 waits `limit_ns` on a barrier that
// nothing arrives on and records kDevTimeoutMma; the other threads wait with
// the full limit and leave as soon as they see the status word set.
__global__ void wait_selftest_kernel(int *err, uint64_t limit_ns, int *left)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_u32(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait(b, 0u, err, kDevTimeoutMma, threadIdx.x == 0 ? limit_ns : kWaitLimitNs);
    if (!ok) atomicAdd(left, 1);
}

// ---------------------------------------------------------------------------
// cta_group::2 variant: a cluster of two CTAs computes a 256 x 256 complex
// tile (inputs i in I2*256 + [0, 256), j in J2*256 + [0, 256), I2 <= J2) with
// M = 256, N = 256 pair MMAs.  CTA r holds the A planes of rows
// I2*256 + r*128 + [0, 128) and the B planes of j rows J2*256 + r*128 + [0, 128);
// each pair MMA reads A rows from both CTAs and B's N halves from both, so a
// CTA supplies half the B operand and the operand bytes per MAC halve.  Per
// 32-sample K step the leader issues
//     Re += A_a B_a^T,  Re += A_b B_b^T,  Im += A_b B_a^T,  Im += (-A_a) B_b^T
// into two 256-column accumulators (all 512 TMEM columns, so the epilogue of
// a tile does not overlap the next tile's MMAs).  Both CTAs' TMA copies
// complete on the leader's barriers; the leader's commits reach both CTAs.
constexpr int kThreads2 = 320;                  // warp 0 TMA, warp 1 MMA + TMEM, warps 2..9 epilogue
constexpr int kEpiThreads2 = 256;               // per CTA
constexpr int kNumBars2 = 2 * kStages + 3;      // full, empty, acc_full, acc_empty, drain
constexpr size_t kSmemBytes2 = 1024 + (size_t)kStages * kStageBytes + kNumBars2 * 8 + 16;

__host__ __device__ constexpr uint32_t make_idesc_m256(bool neg_a)
{
    return (1u << 4) | (neg_a ? (1u << 13) : 0u) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}
constexpr uint32_t kIdesc2 = make_idesc_m256(false);
constexpr uint32_t kIdesc2Neg = make_idesc_m256(true);


__device__ __forceinline__ void tma_load_2d_cg2(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar_cluster)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(bar_cluster)
        : "memory");
}




struct Sched2 {
    int nt2, tiles_per_ch, n_tiles;
    __device__ __forceinline__ void decode(int tile, int &fl, int &I, int &J) const
    {
        fl = tile / tiles_per_ch;
        tile_pair(tile - fl * tiles_per_ch, nt2, I, J);
    }
};

__global__ void __launch_bounds__(kThreads2, 1)
correlate_tc2_kernel(const __grid_constant__ CUtensorMap tmap, const TcArgs a, const Sched2 sc, const int n_k)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    const uint32_t bars = sbase + kStages * kStageBytes;
    auto full_bar = [&](int s) { return bars + 8u * s; };
    auto empty_bar = [&](int s) { return bars + 8u * (kStages + s); };
    const uint32_t accf_bar = bars + 8u * (2 * kStages);
    const uint32_t acce_bar = bars + 8u * (2 * kStages + 1);
    const uint32_t drain_bar = bars + 8u * (2 * kStages + 2);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem_raw + (bars + 8u * kNumBars2 - raw));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    int *err = a.err;
    const int it_begin = (int)(blockIdx.x >> 1), it_step = (int)(gridDim.x >> 1);
    const uint16_t kBoth = 0x3;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        mbar_init(accf_bar, 1);
        mbar_init(acce_bar, 2 * kEpiThreads2);  // both CTAs' epilogue threads
        mbar_init(drain_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&tmap) : "memory");
    }
    if (warp == 1) {  // one collective allocation for the pair: both CTAs issue it
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    cluster_sync();  // the peer's barriers and TMEM exist before anything targets them
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer (both CTAs) ----------------
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int tile = it_begin; ok && tile < sc.n_tiles; tile += it_step) {
                int fl, I2, J2;
                sc.decode(tile, fl, I2, J2);
                const bool diag = (I2 == J2);
                const int rowA = fl * 2 * a.n_pad + I2 * 256 + (int)rank * kTile;
                const int rowB = fl * 2 * a.n_pad + J2 * 256 + (int)rank * kTile;
                for (int kc = 0; kc < n_k; kc++) {
                    if (!mbar_wait(empty_bar(stage), phase ^ 1u, err, kDevTimeoutProducer)) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = sbase + stage * kStageBytes;
                    const uint32_t fb = mapa_rank(full_bar(stage), 0);  // the leader's barrier
                    if (leader) mbar_expect_tx(full_bar(stage), 2u * (diag ? 2 * kPlaneTile : 4 * kPlaneTile));
                    tma_load_2d_cg2(st, &tmap, kc * kKc, rowA, fb);
                    tma_load_2d_cg2(st + kPlaneTile, &tmap, kc * kKc, rowA + a.n_pad, fb);
                    if (!diag) {
                        tma_load_2d_cg2(st + 2 * kPlaneTile, &tmap, kc * kKc, rowB, fb);
                        tma_load_2d_cg2(st + 3 * kPlaneTile, &tmap, kc * kKc, rowB + a.n_pad, fb);
                    }
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
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
            for (int tile = it_begin; ok && tile < sc.n_tiles; tile += it_step) {
                int fl, I2, J2;
                sc.decode(tile, fl, I2, J2);
                const bool diag = (I2 == J2);
                if (!mbar_wait(acce_bar, (uses & 1u) ^ 1u, err, kDevTimeoutMma)) break;
                ++uses;
                fence_after();
                for (int kc = 0; kc < n_k; kc++) {
                    if (!mbar_wait(full_bar(stage), phase, err, kDevTimeoutMma)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t st = sbase + stage * kStageBytes;
                    const uint32_t a_a = st, a_b = st + kPlaneTile;
                    const uint32_t b_a = diag ? a_a : st + 2 * kPlaneTile;
                    const uint32_t b_b = b_a + kPlaneTile;
                    #pragma unroll
                    for (int kk = 0; kk < kKSteps; kk++) {
                        const uint32_t off = kk * 32;
                        const uint32_t acc = (kc != 0 || kk != 0) ? 1u : 0u;
                        mma_f8_cg2(d_re, sw128_desc(a_a + off), sw128_desc(b_a + off), kIdesc2, acc);
                        mma_f8_cg2(d_re, sw128_desc(a_b + off), sw128_desc(b_b + off), kIdesc2, 1u);
                        mma_f8_cg2(d_im, sw128_desc(a_b + off), sw128_desc(b_a + off), kIdesc2, acc);
                        mma_f8_cg2(d_im, sw128_desc(a_a + off), sw128_desc(b_b + off), kIdesc2Neg, 1u);
                    }
                    mma_commit_cg2(empty_bar(stage), kBoth);
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit_cg2(accf_bar, kBoth);
            }
            // Drain: every MMA issued above has finished once this completes.
            mma_commit_cg2(drain_bar, 0x1);
            (void)mbar_wait(drain_bar, 0u, err, kDevTimeoutMma);
        }
    } else {
        // ---------------- epilogue (warps 2..9 of both CTAs) ----------------
        const int q = warp & 3;                 // TMEM lane quadrant this warp may access
        const int half = (warp - 2) >> 2;       // which 128 of the 256 columns
        const int row = q * 32 + lane;
        const uint32_t acce_leader = mapa_rank(acce_bar, 0);
        uint32_t uses = 0;
        const int64_t N = a.N;
        for (int tile = it_begin; tile < sc.n_tiles; tile += it_step) {
            int fl, I2, J2;
            sc.decode(tile, fl, I2, J2);
            const bool ok = mbar_wait(accf_bar, uses & 1u, err, kDevTimeoutEpilogue);
            if (!__all_sync(0xffffffffu, ok)) break;
            ++uses;
            fence_after();
            const int64_t i = (int64_t)I2 * 256 + rank * kTile + row;
            const bool row_ok = i < N;
            const int64_t row_base = i * N - i * (i - 1) / 2 - i;
            int2 *out = reinterpret_cast<int2 *>(a.acc + (int64_t)fl * N * (N + 1));
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16);
            for (int c = half * 128; c < half * 128 + 128; c += 16) {
                uint32_t re[16], im[16];
                tmem_ld16(taddr + c, re);
                tmem_ld16(taddr + 256 + c, im);
                tmem_ld_wait();
                if (row_ok) {
                    const int64_t j0 = (int64_t)J2 * 256 + c;
                    int2 *p = out + row_base + j0;
                    const int64_t e_lo = i - j0, e_hi = N - j0;
                    if (a.accumulate) {
                        int2 old[16];
                        #pragma unroll
                        for (int e = 0; e < 16; e++)
                            if (e >= e_lo && e < e_hi) old[e] = p[e];
                        #pragma unroll
                        for (int e = 0; e < 16; e++)
                            if (e >= e_lo && e < e_hi)
                                p[e] = make_int2(old[e].x + __float2int_rn(__uint_as_float(re[e])),
                                                 old[e].y + __float2int_rn(__uint_as_float(im[e])));
                    } else {
                        #pragma unroll
                        for (int e = 0; e < 16; e++)
                            if (e >= e_lo && e < e_hi)
                                p[e] = make_int2(__float2int_rn(__uint_as_float(re[e])),
                                                 __float2int_rn(__uint_as_float(im[e])));
                    }
                }
            }
            fence_before();
            mbar_arrive_cluster(acce_leader);
        }
    }

    __syncwarp();
    fence_before();
    __syncthreads();
    cluster_sync();  // no copy, commit or arrival of the peer may still target this CTA
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

}  // namespace

cudaError_t launch_correlate_tc(const TcArgs &a, int num_sms, cudaStream_t s)
{
    if (a.nf <= 0) return cudaSuccess;
    if (a.t_pad % kTile != 0 || a.n_pad % kTile != 0 || a.t_pad > kMaxChunkSamples) return cudaErrorInvalidValue;
    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)a.t_pad, (cuuint64_t)a.nf * 2 * a.n_pad};
    const cuuint64_t strides[1] = {(cuuint64_t)a.t_pad};
    const cuuint32_t box[2] = {(cuuint32_t)kKc, kTile};
    const cuuint32_t estr[2] = {1, 1};
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void *)a.planes, dims, strides,
                                        box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                        kKc == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    if (a.sums && (a.n_samples < 1 || a.n_samples > kFusedMaxSamples || a.n_samples > a.t_pad))
        return cudaErrorInvalidValue;
    auto kern = a.sums ? correlate_tc_kernel<false, true> : correlate_tc_kernel<false, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    Sched sc;
    sc.nt = a.n_pad / kTile;
    sc.tiles_per_ch = sc.nt * (sc.nt + 1) / 2;
    sc.n_tiles = a.nf * sc.tiles_per_ch;
    const int grid = sc.n_tiles < num_sms ? sc.n_tiles : num_sms;
    kern<<<grid, kThreads, kSmemBytes, s>>>(map, a, sc, (int)(a.t_pad / kKc), ListArgs{});
    return cudaGetLastError();
}

cudaError_t launch_correlate_tc2(const TcArgs &a, int num_sms, cudaStream_t s)
{
    if (a.nf <= 0) return cudaSuccess;
    if (a.t_pad % kTile != 0 || a.n_pad % 256 != 0 || a.t_pad > kMaxChunkSamples) return cudaErrorInvalidValue;
    CUtensorMap map;
    cudaError_t e = encode_planes_map(&map, a.planes, a.t_pad, (int64_t)a.nf * 2 * a.n_pad);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(correlate_tc2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes2);
    if (e != cudaSuccess) return e;
    Sched2 sc;
    sc.nt2 = a.n_pad / 256;
    sc.tiles_per_ch = sc.nt2 * (sc.nt2 + 1) / 2;
    sc.n_tiles = a.nf * sc.tiles_per_ch;
    const int clusters = sc.n_tiles < num_sms / 2 ? sc.n_tiles : num_sms / 2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * clusters, 1, 1);
    cfg.blockDim = dim3(kThreads2, 1, 1);
    cfg.dynamicSmemBytes = kSmemBytes2;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, correlate_tc2_kernel, map, a, sc, (int)(a.t_pad / kKc));
}

cudaError_t encode_planes_map(CUtensorMap *map, const uint8_t *planes, int64_t t_pad, int64_t rows)
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)t_pad, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)t_pad};
    const cuuint32_t box[2] = {(cuuint32_t)kKc, kTile};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void *)planes, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, kKc == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t selftest_wait_timeout(int64_t limit_ns, int *status, int *left)
{
    int *d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * sizeof(int));
    if (e != cudaSuccess) return e;
    e = cudaMemset(d, 0, 2 * sizeof(int));
    if (e == cudaSuccess) {
        wait_selftest_kernel<<<1, 64>>>(d, (uint64_t)limit_ns, d + 1);
        e = cudaGetLastError();
    }
    int h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    *status = h[0];
    *left = h[1];
    return e;
}

cudaError_t prepare_correlate_tc_listed()
{
    return cudaFuncSetAttribute(correlate_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSmemBytes);
}

cudaError_t launch_correlate_tc_listed(const ListArgs &L, int grid, cudaStream_t s)
{
    if (grid <= 0) return cudaSuccess;
    CUtensorMap unused;
    memset(&unused, 0, sizeof(unused));
    TcArgs a{};
    Sched sc{};
    correlate_tc_kernel<true><<<grid, kThreads, kSmemBytes, s>>>(unused, a, sc, 0, L);
    return cudaGetLastError();
}

}  // namespace xeng
