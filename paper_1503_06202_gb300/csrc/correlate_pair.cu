// correlate_pair.cu -- the X-engine step for many inputs in one pass over the
// raw bytes: the nibble split (paper Sec. II-A) fused into the Hermitian
// correlation (Sec. IV-C-1, Eq. 1), with no decoded planes in HBM.
//
// A cluster of two CTAs owns one upper-triangle pair (I2 <= J2) of 256-input
// blocks of one channel at a time, channel-major and round-robin over the
// clusters (the clusters at work share one or two channels' raw bytes in L2).
// The A operand is the column block: CTA r takes A inputs j = J2*256 + r*128 +
// [0, 128) and B inputs i = I2*256 + r*128 + [0, 128), so a CTA's TMEM lanes
// are inputs j and its columns inputs i.  Per stage of kPKc (128) samples its
// producer TMA-loads those two raw tiles (one on the diagonal, where A = B)
// with a 128-byte swizzle -- the canonical MN-major layout of an 8-bit tcgen05
// operand -- into a raw ring; its converter warps split each byte at its own
// offset into the Im and Re planes of a plane stage and sum each input's
// nibbles.  The leader issues cta_group::2 MMAs of M = 256, N = 256 over the
// pair's planes:
//     Re += A_re B_re^T + A_im B_im^T,   Im += A_re B_im^T + (-A_im) B_re^T
// which with A = x_j, B = x_i is Im of x_i conj(x_j) (each CTA supplies its
// 128 rows of A and its half of B, so per MMA a CTA reads 8 KB of operands for
// 128 x 256 x 32 multiply-adds; per stage it converts two 16 KB tiles for 16
// MMAs, about 2048 tensor cycles).  The 256 x 256 complex accumulator fills
// all 512 TMEM columns of both CTAs; the epilogue (tcgen05.ld -> int32
// triangle) follows each pair and cannot overlap the next pair's MMAs, so its
// stores are laid out for the memory system: per column i, a warp's 32 lanes
// hold 32 consecutive inputs j, one 256-byte run of the triangle's row i
// (8-byte aligned whatever the row's start, unlike a row's 8-pair chunks).
//
// The stage length sets the cost: a stage carries a fixed cost (barrier round
// trips, the proxy fence, the ring hand-offs) beside its conversion work, so
// 128-sample stages in two plane stages and two raw slots measured faster on
// GB300 than 64-sample stages in four and five (full CHIME, 2048 inputs x 1024
// channels x 8192 samples: 43.5 ms against 61 ms).
//
// The planes hold raw nibbles: a byte whose low four bits are u (0..15) and
// whose high four bits are clear is the FP8 E4M3 code of u / 512.  With p, q
// the Re and Im nibbles and x = (p - 8) + i (q - 8), over a launch of n samples
//     Re V_ij = sum(p_i p_j + q_i q_j) - 8 (S_i + S_j) + 128 n,
//     Im V_ij = sum(q_i p_j - p_i q_j) + 8 (D_i - D_j),
// with S = P + Q, D = P - Q and P, Q the sums of an input's nibbles.  Each
// CTA's converters form the sums of its A and B tiles per pair; the B sums go
// to both CTAs (the epilogue of a row needs all 256 columns').  The MMA sums
// are integers / 2^18 of at most 450 n; launches of at most 32,768 samples
// keep them below 2^24, exact in f32.
//
// Roles per CTA (576 threads):
//   warp 0       TMA producer: raw tiles into the raw ring
//   warp 1       TMEM allocation (collective for the pair); MMA issuer (leader)
//   warps 2..9   converters: raw slot -> Im and Re planes of a plane stage, nibble sums;
//                four warps a tile, all eight on the one tile of a diagonal pair
//                (each thread half its chunks: 41.8-42.2 ms for full CHIME
//                against 42.9 with the B tile's warps idle there)
//   warps 10..17 epilogue: TMEM -> packed int32 triangle, two warps per TMEM lane
//                quadrant taking alternate 8-column chunks (so both have work on
//                diagonal pairs, where only the columns up to a lane's input count),
//                each loading its next chunk from TMEM under the current one's stores
#include <cstring>

#include "tc_ptx.cuh"
#include "xeng_internal.h"

namespace xeng {
namespace {

// Samples per stage (a build parameter, 64 or 128), plane stages and raw slots.
#ifndef XENG_PAIR_KC
#define XENG_PAIR_KC 128
#endif
constexpr int kPKc = XENG_PAIR_KC;          // samples per stage
static_assert(kPKc == 64 || kPKc == 128, "64 or 128 samples per stage");
constexpr int kPBox = kPKc * 128;           // one raw tile or plane tile: kPKc samples x 128 inputs
constexpr int kPRawBytes = 2 * kPBox;       // raw slot: the CTA's A and B tiles
constexpr int kPPlaneBytes = 4 * kPBox;     // plane stage: A_im, A_re, B_im, B_re
#ifndef XENG_PAIR_PLANE_STAGES
#define XENG_PAIR_PLANE_STAGES (4 * 64 / XENG_PAIR_KC)
#endif
#ifndef XENG_PAIR_RAW_SLOTS
#define XENG_PAIR_RAW_SLOTS (XENG_PAIR_KC == 128 ? 2 : 5)
#endif
constexpr int kPPlanes = XENG_PAIR_PLANE_STAGES, kPRaws = XENG_PAIR_RAW_SLOTS;
constexpr int kPConvWarp0 = 2, kPConvWarps = 8;
// Epilogue warps: a multiple of four (each TMEM lane quadrant gets the same
// number, which split its 256 columns in interleaved 8-column chunks).  Measured
// on GB300, full CHIME: 8 warps 41.7 ms; 12 or 16 (fewer registers a thread,
// some spilled) 44.5; 4 (116 registers, no spills) 1% slower than 8 on one box;
// with the chunk-ahead epilogue, 4 (123 registers) 41.58-42.32 against
// 41.55-41.72 for 8 on one box.
// Each quadrant's columns as two halves instead: 42.8.
#ifndef XENG_PAIR_EPI_WARPS
#define XENG_PAIR_EPI_WARPS 8
#endif
constexpr int kPEpiWarp0 = kPConvWarp0 + kPConvWarps, kPEpiWarps = XENG_PAIR_EPI_WARPS;
static_assert(kPEpiWarps % 4 == 0 && kPEpiWarps >= 4, "epilogue warps: a multiple of four");
constexpr int kPEpiPerQuad = kPEpiWarps / 4;
constexpr int kPThreads = 32 * (kPEpiWarp0 + kPEpiWarps);
constexpr uint32_t kPTmemCols = 512;
constexpr int kPSums = 2 * 384 * 8;     // per item parity: (P, Q) of the CTA's A rows, then all 256 B columns
constexpr int kPScratch = 2 * 4 * 128 * 8;  // per tile and warp of it: (P, Q) partials of its 128 inputs
// barriers: raw full and empty per slot, plane full and empty per stage; acc
// full, acc empty, drain; sums full and empty per parity
constexpr int kPBars = 2 * kPRaws + 2 * kPPlanes + 3 + 4;
constexpr size_t kPSmem = 1024 + (size_t)kPPlanes * kPPlaneBytes + (size_t)kPRaws * kPRawBytes + kPSums + kPScratch +
                          kPBars * 8 + 16;
static_assert(kPSmem <= 232448, "shared memory over the per-CTA limit");
constexpr int kPChunks = 2 * kPBox / 16 / (32 * kPConvWarps);

constexpr int kPWiden = 16 / kPChunks;

// Instruction descriptor, kind::f8f6f4: D f32, A and B E4M3, both MN-major
// (bits 15, 16), N = 256, M = 256; bit 13 negates A.
__host__ __device__ constexpr uint32_t pair_idesc(bool neg_a)
{
    return (1u << 4) | (neg_a ? (1u << 13) : 0u) | (1u << 15) | (1u << 16) | ((uint32_t)(256 >> 3) << 17) |
           ((uint32_t)(256 >> 4) << 24);
}

// MN-major operand with a 128-byte swizzle: rows of 128 elements along M/N,
// 8-row groups along K 1 KB apart (stride byte offset), version 1.  A CTA's
// operand is one atom wide along M/N, so the leading byte offset is not used.
__device__ __forceinline__ uint64_t pdesc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(kPBox >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

struct PairArgs {
    int64_t t0, nt;          // samples t0 .. t0 + nt - 1 of the block, nt <= kFusedMaxSamples
    int32_t F, N, f0, nf;    // channels f0 .. f0 + nf - 1
    int32_t nt2;             // 256-input blocks
    int32_t pairs_per_ch;    // nt2 (nt2 + 1) / 2
    int32_t n_items;         // nf * pairs_per_ch
    int32_t *acc;            // [nf][N(N+1)/2][2], channel f0 + fl at fl
    int accumulate;          // 0: store, 1: add
    int *err;
    const CUtensorMap *maps;  // null: raw_map over one block; else a map per block of spb stages,
    int32_t spb;              // the launch's samples running through the blocks in order
    const PairJob *jobs;      // listed launches: the jobs (items job after job), else unused
    int32_t n_jobs;
};

struct PairItem {
    int fl, I2, J2;
    int job;  // listed launches
};

// Item `it`: channel-major, the channel's block pairs I2 <= J2 row by row; in a
// listed launch first the job whose items hold `it` (the last with item0 <= it).
template <bool kListed>
__device__ __forceinline__ PairItem pair_item(const PairArgs &a, int it)
{
    PairItem w;
    int local = it, ppc = a.pairs_per_ch, nt2 = a.nt2;
    w.job = 0;
    if (kListed) {
        int lo = 0, hi = a.n_jobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.jobs[mid].item0 <= it) lo = mid;
            else hi = mid - 1;
        }
        w.job = lo;
        local = it - a.jobs[lo].item0;
        ppc = a.jobs[lo].pairs_per_ch;
        nt2 = a.jobs[lo].nt2;
    }
    w.fl = local / ppc;
    int r = local - w.fl * ppc, i = 0;
    while (r >= nt2 - i) {
        r -= nt2 - i;
        ++i;
    }
    w.I2 = i;
    w.J2 = i + r;
    return w;
}

// kAdd: the launch adds to the triangle (a later piece of an integration)
// instead of storing it; a separate instantiation, so the storing epilogue
// keeps two chunks' TMEM words in registers without spilling.
template <bool kListed, bool kAdd>
__global__ void __launch_bounds__(kPThreads, 1)
correlate_pair_kernel(const __grid_constant__ CUtensorMap raw_map, const PairArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t *sgen = smem_raw + (sbase - raw);
    // plane stages first, then the raw slots, the item sums, the scratch and the barriers
    const uint32_t raw0 = sbase + kPPlanes * kPPlaneBytes;
    const uint32_t sums_u = raw0 + kPRaws * kPRawBytes;
    const uint32_t scratch_u = sums_u + kPSums;
    const uint32_t bars = scratch_u + kPScratch;
    int2 *sums = reinterpret_cast<int2 *>(sgen + (sums_u - sbase));        // [parity][384] (P, Q)
    int2 *scratch = reinterpret_cast<int2 *>(sgen + (scratch_u - sbase));  // [tile][warp of tile][128] (P, Q)
    auto plane = [&](int s) { return sbase + (uint32_t)(s * kPPlaneBytes); };
    auto slot = [&](int s) { return raw0 + (uint32_t)(s * kPRawBytes); };
    auto rawf = [&](int s) { return bars + 8u * s; };
    auto rawe = [&](int s) { return bars + 8u * (kPRaws + s); };
    auto full = [&](int s) { return bars + 8u * (2 * kPRaws + s); };
    auto empty = [&](int s) { return bars + 8u * (2 * kPRaws + kPPlanes + s); };
    const uint32_t accf = bars + 8u * (2 * kPRaws + 2 * kPPlanes);
    const uint32_t acce = accf + 8u;
    const uint32_t drain = accf + 16u;
    auto sums_full = [&](int par) { return accf + 24u + 8u * par; };
    auto sums_empty = [&](int par) { return accf + 40u + 8u * par; };
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem_raw + (bars + 8u * kPBars - raw));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const uint32_t peer = rank ^ 1u;
    const bool leader = rank == 0;
    int *err = a.err;
    const int it_begin = (int)(blockIdx.x >> 1), it_step = (int)(gridDim.x >> 1);
    const int n_k = (int)((a.nt + kPKc - 1) / kPKc);
    const uint16_t kBoth = 0x3;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kPRaws; s++) {
            mbar_init(rawf(s), 1);
            mbar_init(rawe(s), kPConvWarps);      // this CTA's converter warps
        }
        for (int s = 0; s < kPPlanes; s++) {
            mbar_init(full(s), 2 * kPConvWarps);  // the leader's: both CTAs' converter warps
            mbar_init(empty(s), 1);
        }
        mbar_init(accf, 1);
        mbar_init(acce, 2 * kPEpiWarps);          // the leader's: both CTAs' epilogue warps
        mbar_init(drain, 1);
        for (int par = 0; par < 2; par++) {
            mbar_init(sums_full(par), 2 * kPConvWarps);  // both CTAs' converter warps (B sums from both)
            mbar_init(sums_empty(par), 2 * kPEpiWarps);  // both CTAs' epilogue warps (they read these B sums)
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&raw_map) : "memory");
    }
    if (warp == 1) {  // one collective allocation for the pair: both CTAs issue it
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kPTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    cluster_sync();  // the peer's barriers and TMEM exist before anything targets them
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer (both CTAs: each its own tiles) ----------------
            int s = 0, issued = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int it = it_begin; ok && it < a.n_items; it += it_step) {
                const PairItem w = pair_item<kListed>(a, it);
                const int f = kListed ? w.fl : a.f0 + w.fl;
                const int nk = kListed ? a.jobs[w.job].n_k : n_k;
                const bool diag = w.I2 == w.J2;
                const int xa = w.J2 * 256 + (int)rank * 128, xb = w.I2 * 256 + (int)rank * 128;
                for (int kc = 0; kc < nk; kc++) {
                    if (!mbar_try_wait(rawe(s), ph ^ 1u) && !mbar_wait(rawe(s), ph ^ 1u, err, kDevTimeoutProducer)) {
                        ok = false;
                        break;
                    }
                    const CUtensorMap *mp = &raw_map;
                    int z = (int)(a.t0 + (int64_t)kc * kPKc);
                    if (kListed) {  // the job's own map
                        mp = a.jobs[w.job].map;
                        z = kc * kPKc;
                    } else if (a.maps) {  // blocks of spb stages, each with its own map
                        mp = a.maps + kc / a.spb;
                        z = (kc % a.spb) * kPKc;
                    }
                    mbar_expect_tx(rawf(s), diag ? kPBox : kPRawBytes);
                    tma_load_3d(slot(s), mp, xa, f, z, rawf(s));
                    if (!diag) tma_load_3d(slot(s) + kPBox, mp, xb, f, z, rawf(s));
                    ++issued;
                    if (++s == kPRaws) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (!ok) {
                // Let the copies already issued land before the CTA can exit.
                for (int k = 1; k <= kPRaws && k <= issued; k++) {
                    int sk = s - k, p = (int)ph;
                    if (sk < 0) { sk += kPRaws; p ^= 1; }
                    (void)mbar_wait(rawf(sk), (uint32_t)p, err, kDevTimeoutProducer);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            // ---------------- MMA issuer (leader CTA) ----------------
            int s = 0;
            uint32_t ph = 0, uses = 0;
            bool ok = true;
            const uint32_t d_re = tmem, d_im = tmem + 256u;
            for (int it = it_begin; ok && it < a.n_items; it += it_step) {
                const PairItem w = pair_item<kListed>(a, it);
                const bool diag = w.I2 == w.J2;
                const int nk = kListed ? a.jobs[w.job].n_k : n_k;
                if (!mbar_wait(acce, (uses & 1u) ^ 1u, err, kDevTimeoutMma)) break;
                ++uses;
                fence_after();
                for (int kc = 0; kc < nk; kc++) {
                    if (!mbar_try_wait(full(s), ph) && !mbar_wait_cluster(full(s), ph, err, kDevTimeoutMma)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t st = plane(s);
                    const uint64_t dai = pdesc(st), dar = pdesc(st + kPBox);
                    const uint64_t dbi = diag ? dai : pdesc(st + 2 * kPBox);
                    const uint64_t dbr = diag ? dar : pdesc(st + 3 * kPBox);
                    #pragma unroll
                    for (int kk = 0; kk < kPKc / 32; kk++) {  // +32 samples = +4 KB = +256 in the address field
                        const uint32_t acc = (kc != 0 || kk != 0) ? 1u : 0u;
                        const uint64_t k4 = 256u * kk;
                        mma_f8_cg2(d_re, dar + k4, dbr + k4, pair_idesc(false), acc);
                        mma_f8_cg2(d_re, dai + k4, dbi + k4, pair_idesc(false), 1u);
                        mma_f8_cg2(d_im, dar + k4, dbi + k4, pair_idesc(false), acc);
                        mma_f8_cg2(d_im, dai + k4, dbr + k4, pair_idesc(true), 1u);
                    }
                    mma_commit_cg2(empty(s), kBoth);
                    if (++s == kPPlanes) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit_cg2(accf, kBoth);
            }
            // Drain: every MMA issued above has finished once this completes.
            mma_commit_cg2(drain, 0x1);
            (void)mbar_wait(drain, 0u, err, kDevTimeoutMma);
        }
    } else if (warp < kPEpiWarp0) {
        // ---------------- converters (both CTAs) ----------------
        // Thread u (0..255) takes tile g = u / 128 (A, then B) and, in it, the
        // 16-byte chunks v + 128 k (v = u % 128, k = 0..kPChunks-1): sample rows
        // v / 8 + 16 k, physical chunk v % 8 -- a quarter-warp covers one whole
        // 128-byte row, so the accesses are bank-conflict-free.  The rows' swizzle
        // (chunk ^ row % 8) is the same for all of them, so the thread always
        // holds the same 16 inputs: logical chunk lc = (v % 8) ^ (v / 8 % 8).
        // Its nibble sums run in bytes (kPChunks x kPWiden x 15 <= 240 between
        // widenings), then in 16-bit lanes (nt / 16 rows x 15 <= 30,720).
        const int u = (warp - kPConvWarp0) * 32 + lane;
        const int g = u >> 7, v = u & 127;
        const int r0 = v >> 3, lc = (v & 7) ^ (r0 & 7);
        const int wt = (u >> 5) & 3;                               // warp within the tile
        const uint32_t roff = (uint32_t)(g * kPBox + v * 16);      // in a raw slot (+ 2048 k)
        const uint32_t poff = (uint32_t)(2 * g * kPBox + v * 16);  // Im plane of the tile (+ 2048 k; Re kPBox on)
        const uint32_t full_leader = mapa_rank(full(0), 0) - full(0);  // offset into the leader's window
        const int nt = (int)a.nt;                                  // <= kFusedMaxSamples
        int rs = 0, ps = 0, local = 0;
        uint32_t rph = 0, pph = 0;
        for (int it = it_begin; it < a.n_items; it += it_step, ++local) {
            const PairItem w = pair_item<kListed>(a, it);
            const bool diag = w.I2 == w.J2;
            // The diagonal has the A tile only (B = A): there both tiles' threads
            // split it, the B tile's threads taking its second half of chunks.
            const int nch = diag ? kPChunks / 2 : kPChunks;  // chunks of this thread
            const int kofs = diag ? g * (kPChunks / 2) : 0;  // its first chunk
            const uint32_t roff_w = diag ? (uint32_t)(v * 16 + 2048 * kofs) : roff;
            const uint32_t poff_w = diag ? (uint32_t)(v * 16 + 2048 * kofs) : poff;
            const int nk = kListed ? a.jobs[w.job].n_k : n_k;
            const int nt_w = kListed ? a.jobs[w.job].nt : nt;  // samples of the item's launch
            bool ok = true;
            uint32_t pb[4] = {0, 0, 0, 0}, qb[4] = {0, 0, 0, 0};
            uint32_t P16[8] = {0, 0, 0, 0, 0, 0, 0, 0}, Q16[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            auto widen = [&]() {
                #pragma unroll
                for (int k = 0; k < 4; k++) {
                    P16[2 * k] += pb[k] & 0x00FF00FFu;
                    P16[2 * k + 1] += (pb[k] >> 8) & 0x00FF00FFu;
                    Q16[2 * k] += qb[k] & 0x00FF00FFu;
                    Q16[2 * k + 1] += (qb[k] >> 8) & 0x00FF00FFu;
                    pb[k] = qb[k] = 0;
                }
            };
            for (int kc = 0; kc < nk; kc++) {
                ok = mbar_wait_backoff(rawf(rs), rph, err, kDevTimeoutProducer, XENG_CONV_SLEEP_NS);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                const int rows_left = nt_w - kc * kPKc;  // samples of this stage inside the launch (may exceed kPKc)
                const uint8_t *src = sgen + (slot(rs) - sbase) + roff_w;
                uint4 x[kPChunks];
                #pragma unroll
                for (int k = 0; k < kPChunks; k++) {
                    x[k] = k < nch ? *reinterpret_cast<const uint4 *>(src + 2048 * k) : make_uint4(0, 0, 0, 0);
                    if (r0 + 16 * (k + kofs) >= rows_left) x[k] = make_uint4(0, 0, 0, 0);  // past the launch: adds nothing
                }
                // the raw slot goes back with the plane stage, once the plane stores
                // (which consume the loaded words) are done
                const int rcur = rs;
                if (++rs == kPRaws) {
                    rs = 0;
                    rph ^= 1u;
                }
                ok = mbar_wait_backoff(empty(ps), pph ^ 1u, err, kDevTimeoutProducer, XENG_CONV_SLEEP_NS);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                uint8_t *dim = sgen + (plane(ps) - sbase) + poff_w;  // Im plane of the tile
                uint8_t *dre = dim + kPBox;                          // Re plane of the tile
                #pragma unroll
                for (int k = 0; k < kPChunks; k++) {
                    if (k >= nch) break;
                    uint4 re, im;
                    re.x = (x[k].x >> 4) & 0x0F0F0F0Fu;
                    re.y = (x[k].y >> 4) & 0x0F0F0F0Fu;
                    re.z = (x[k].z >> 4) & 0x0F0F0F0Fu;
                    re.w = (x[k].w >> 4) & 0x0F0F0F0Fu;
                    im.x = x[k].x & 0x0F0F0F0Fu;
                    im.y = x[k].y & 0x0F0F0F0Fu;
                    im.z = x[k].z & 0x0F0F0F0Fu;
                    im.w = x[k].w & 0x0F0F0F0Fu;
                    *reinterpret_cast<uint4 *>(dre + 2048 * k) = re;
                    *reinterpret_cast<uint4 *>(dim + 2048 * k) = im;
                    pb[0] += re.x; pb[1] += re.y; pb[2] += re.z; pb[3] += re.w;
                    qb[0] += im.x; qb[1] += im.y; qb[2] += im.z; qb[3] += im.w;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // planes visible to the MMAs
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive_cluster(full(ps) + full_leader);
                    mbar_arrive(rawe(rcur));
                }
                if (++ps == kPPlanes) {
                    ps = 0;
                    pph ^= 1u;
                }
                if ((kc + 1) % kPWiden == 0) widen();
            }
            // End of the pair: every converter warp reaches the barriers below, failed
            // or not, and they OR the failures, so the warps leave together.
            if (ok) {
                widen();
                // the four lanes of a warp holding the same inputs (rows differing in
                // their two low bits: lanes ^ 9, ^ 18) add up -- two in 16-bit lanes
                // (<= 2 x 15 x 2048), the other two in 32 bits -- and one of them
                // writes the warp's partials; input 4w + b is byte b of word w
                #pragma unroll
                for (int k = 0; k < 8; k++) {
                    P16[k] += __shfl_xor_sync(0xffffffffu, P16[k], 9);
                    Q16[k] += __shfl_xor_sync(0xffffffffu, Q16[k], 9);
                }
                #pragma unroll
                for (int m = 0; m < 16; m++) {
                    const int wd = m >> 2, b = m & 3;
                    uint32_t pv = (P16[2 * wd + (b & 1)] >> (16 * (b >> 1))) & 0xFFFFu;
                    uint32_t qv = (Q16[2 * wd + (b & 1)] >> (16 * (b >> 1))) & 0xFFFFu;
                    pv += __shfl_xor_sync(0xffffffffu, pv, 18);
                    qv += __shfl_xor_sync(0xffffffffu, qv, 18);
                    if ((r0 & 3) == 0) scratch[(g * 4 + wt) * 128 + lc * 16 + m] = make_int2((int)pv, (int)qv);
                }
            }
            bool fail = bar_any(1, kPConvWarps * 32, !ok);
            if (!fail) {
                // thread u totals input u % 128 of tile g over the tile's four warps;
                // the buffer was last read by both CTAs' epilogues two pairs ago
                const int par = local & 1;
                const int k = v;
                ok = mbar_wait_cluster(sums_empty(par), (uint32_t)((local >> 1) & 1) ^ 1u, err, kDevTimeoutProducer);
                if (__all_sync(0xffffffffu, ok)) {
                    const int tg = diag ? 0 : g;  // on the diagonal the B sums are the A sums
                    int P = 0, Q = 0;
                    #pragma unroll
                    for (int q4 = 0; q4 < 4; q4++) {
                        const int2 p2 = scratch[(tg * 4 + q4) * 128 + k];
                        P += p2.x;
                        Q += p2.y;
                    }
                    if (diag) {  // the A tile's other chunks, summed by the B tile's threads
                        #pragma unroll
                        for (int q4 = 0; q4 < 4; q4++) {
                            const int2 p2 = scratch[(4 + q4) * 128 + k];
                            P += p2.x;
                            Q += p2.y;
                        }
                    }
                    int2 *sp = sums + par * 384;
                    if (g == 0) {
                        sp[k] = make_int2(P, Q);  // this CTA's A rows
                    } else {
                        // this CTA's half of the B columns, here and in the peer
                        const int col = 128 + (int)rank * 128 + k;
                        sp[col] = make_int2(P, Q);
                        st_cluster_v2(mapa_rank(sums_u + (uint32_t)((par * 384 + col) * 8), peer), P, Q);
                    }
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive_cluster(mapa_rank(sums_full(par), rank));
                        mbar_arrive_cluster(mapa_rank(sums_full(par), peer));
                    }
                } else {
                    ok = false;
                }
            }
            // the scratch may be rewritten (next pair) once every reading thread is done
            fail = bar_any(1, kPConvWarps * 32, !ok) || fail;
            if (fail) break;
        }
    } else {
        // ---------------- epilogue (both CTAs) ----------------
        const int q = warp & 3;                          // TMEM lane quadrant this warp may access
        const int cbeg = 8 * ((warp - kPEpiWarp0) >> 2);  // this warp's first column; then every 8 * kPEpiPerQuad
        const int row = q * 32 + lane;
        const uint32_t acce_leader = mapa_rank(acce, 0);
        uint32_t uses = 0;
        int local = 0;
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16);
        for (int it = it_begin; it < a.n_items; it += it_step, ++local) {
            const PairItem w = pair_item<kListed>(a, it);
            const int N = kListed ? a.jobs[w.job].N : a.N;  // <= 4096: triangle offsets within a channel fit in int
            const int n128 = 128 * (kListed ? a.jobs[w.job].nt : (int)a.nt);  // 64 n from each of the two products
            int32_t *const acc = kListed ? a.jobs[w.job].acc : a.acc;
            const int par = local & 1;
            bool ok = mbar_wait_backoff(accf, uses & 1u, err, kDevTimeoutEpilogue, 128);
            ok = ok && mbar_wait_cluster(sums_full(par), (uint32_t)((local >> 1) & 1), err, kDevTimeoutEpilogue);
            // the barrier ORs the eight warps' failures, so they leave together
            if (bar_any(2, kPEpiWarps * 32, !ok)) break;
            ++uses;
            fence_after();
            const int j_warp = w.J2 * 256 + (int)rank * 128 + q * 32;  // the warp's first input j
            const int j = j_warp + lane;
            const bool lane_ok = j < N;
            int2 *out = reinterpret_cast<int2 *>(acc) + (int64_t)w.fl * ((int64_t)N * (N + 1) / 2);
            const int2 *sp = sums + par * 384;
            const int2 pq = sp[row];  // this lane's input j (A rows of this CTA)
            const int sj = pq.x + pq.y, dj = pq.x - pq.y;
            const int2 *cs = sp + 128;  // inputs i of the 256 columns
            const int ibase = w.I2 * 256;
            // Corrects the chunk of columns c..c+7 held in (vre, vim) in place and stores it.
            auto put_chunk = [&](const int c, uint32_t (&vre)[8], uint32_t (&vim)[8], const bool add) {
                const int i0 = ibase + c;
                #pragma unroll
                for (int e = 0; e < 8; e++) {  // corrected values in place of the accumulator words
                    const int2 pi = cs[c + e];  // the same for every lane: a broadcast
                    // accumulators hold integer sums / 2^18: x 2^18 is exact
                    vre[e] = (uint32_t)(__float2int_rn(262144.0f * __uint_as_float(vre[e])) -
                                        8 * (sj + pi.x + pi.y) + n128);
                    vim[e] = (uint32_t)(__float2int_rn(262144.0f * __uint_as_float(vim[e])) +
                                        8 * ((pi.x - pi.y) - dj));
                }
                // pair (i, j) sits at i*N - i*(i-1)/2 + (j - i) in the channel's triangle;
                // pair (i + 1, j) is N - i - 1 entries further on
                const int off0 = i0 * N - i0 * (i0 - 1) / 2 - i0 + j;
                const int last = min(j - i0, N - 1 - i0);  // elements e <= last are pairs of the triangle
                if (add) {
                    int2 o[8];
                    int off = off0;
                    #pragma unroll
                    for (int e = 0; e < 8; e++) {
                        if (lane_ok && e <= last) o[e] = __ldcs(out + off);
                        off += N - (i0 + e) - 1;
                    }
                    off = off0;
                    #pragma unroll
                    for (int e = 0; e < 8; e++) {
                        if (lane_ok && e <= last) __stcs(out + off, make_int2(o[e].x + (int)vre[e], o[e].y + (int)vim[e]));
                        off += N - (i0 + e) - 1;
                    }
                } else {
                    int off = off0;
                    #pragma unroll
                    for (int e = 0; e < 8; e++) {
                        if (lane_ok && e <= last) __stcs(out + off, make_int2((int)vre[e], (int)vim[e]));
                        off += N - (i0 + e) - 1;
                    }
                }
            };
            // warp-uniform: columns inside the channel and up to some lane's diagonal
            auto chunk_ok = [&](const int c) { return c < 256 && ibase + c < N && ibase + c <= j_warp + 31; };
            constexpr int kStep = 8 * kPEpiPerQuad;
            if (kAdd && j_warp < N) {  // adding to the triangle: one chunk at a time
                for (int c = cbeg; chunk_ok(c); c += kStep) {
                    uint32_t vre[8], vim[8];
                    tmem_ld8(taddr + c, vre);
                    tmem_ld8(taddr + 256 + c, vim);
                    tmem_ld_wait();
                    put_chunk(c, vre, vim, true);
                }
            } else if (j_warp < N) {
                // two register sets: the next chunk's TMEM loads run under this chunk's stores
                // (full CHIME, same box: 40.6-41.7 ms against 42.8-42.9 one chunk at a time)
                uint32_t ra[8], ia[8], rb[8], ib[8];
                int c = cbeg;
                if (chunk_ok(c)) {
                    tmem_ld8(taddr + c, ra);
                    tmem_ld8(taddr + 256 + c, ia);
                }
                tmem_ld_wait();
                while (chunk_ok(c)) {
                    const int c1 = c + kStep;
                    const bool ok1 = chunk_ok(c1);
                    if (ok1) {
                        tmem_ld8(taddr + c1, rb);
                        tmem_ld8(taddr + 256 + c1, ib);
                    }
                    put_chunk(c, ra, ia, false);
                    tmem_ld_wait();
                    if (!ok1) break;
                    const int c2 = c1 + kStep;
                    const bool ok2 = chunk_ok(c2);
                    if (ok2) {
                        tmem_ld8(taddr + c2, ra);
                        tmem_ld8(taddr + 256 + c2, ia);
                    }
                    put_chunk(c1, rb, ib, false);
                    tmem_ld_wait();
                    c = c2;
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive_cluster(acce_leader);
                // this CTA's reads of both CTAs' sums are done for this parity
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
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPTmemCols));
    }
}

}  // namespace

bool pair_ok(const uint8_t *block, int32_t N)
{
    return N >= 16 && N <= 4096 && N % 16 == 0 && (reinterpret_cast<uintptr_t>(block) & 15) == 0;
}

cudaError_t encode_pair_map(CUtensorMap *map, const uint8_t *block, int64_t T_block, int32_t F, int32_t N)
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    // raw block: dims (input, channel, sample), boxes of 128 inputs x 1 channel x kPKc
    // samples with a 128-byte swizzle (the MN-major operand layout); inputs past N and
    // samples past the block read as zero bytes, nibbles 0 that add nothing (the
    // converters zero the samples past the launch; rows and columns past N are never
    // written)
    cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)F, (cuuint64_t)T_block};
    cuuint64_t strides[2] = {(cuuint64_t)N, (cuuint64_t)N * F};
    cuuint32_t box[3] = {128, 1, (cuuint32_t)kPKc}, estr[3] = {1, 1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, (void *)block, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

int pair_stage_samples() { return kPKc; }

cudaError_t launch_correlate_pair(const uint8_t *block, int64_t T_block, int64_t t0, int64_t nt, int32_t F, int32_t N,
                                  int32_t f0, int32_t nf, int32_t *acc, int accumulate, int *err, int num_sms,
                                  cudaStream_t s,
                                  const CUtensorMap *maps, int32_t spb)
{
    if (nf <= 0 || nt <= 0) return cudaSuccess;
    if (!pair_ok(maps ? nullptr : block, N) || (maps && (spb < 1 || t0 != 0)) || nt > kFusedMaxSamples ||
        t0 < 0 || t0 + nt > T_block || T_block > 2147483647LL ||
        f0 < 0 || f0 + nf > F || num_sms < 2 || (reinterpret_cast<uintptr_t>(acc) & 7) != 0)
        return cudaErrorInvalidValue;
    const int32_t nt2 = (N + 255) / 256;
    const int64_t n_items = (int64_t)nf * (nt2 * (nt2 + 1) / 2);
    if (n_items > 2147483647LL) return cudaErrorInvalidValue;
    CUtensorMap map;
    if (maps) {
        memset(&map, 0, sizeof map);  // not read: the stages take the blocks' maps
    } else {
        cudaError_t e0 = encode_pair_map(&map, block, T_block, F, N);
        if (e0 != cudaSuccess) return e0;
    }
    auto kernel = accumulate ? correlate_pair_kernel<false, true> : correlate_pair_kernel<false, false>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPSmem);
    if (e != cudaSuccess) return e;
    PairArgs a;
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
    a.accumulate = accumulate;
    a.err = err;
    a.maps = maps;
    a.spb = spb;
    const int64_t clusters = n_items < num_sms / 2 ? n_items : num_sms / 2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * clusters), 1, 1);
    cfg.blockDim = dim3(kPThreads, 1, 1);
    cfg.dynamicSmemBytes = kPSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    a.jobs = nullptr;
    a.n_jobs = 0;
    return cudaLaunchKernelEx(&cfg, kernel, map, a);
}

cudaError_t launch_correlate_pair_listed(const PairJob *jobs, int32_t n_jobs, int64_t n_items, int *err, int num_sms,
                                         cudaStream_t s)
{
    if (n_jobs <= 0 || n_items <= 0) return cudaSuccess;
    if (!jobs || num_sms < 2 || n_items > 2147483647LL) return cudaErrorInvalidValue;
    cudaError_t e =
        cudaFuncSetAttribute(correlate_pair_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPSmem);
    if (e != cudaSuccess) return e;
    CUtensorMap unused;
    memset(&unused, 0, sizeof unused);  // not read: every item takes its job's map
    PairArgs a;
    memset(&a, 0, sizeof a);
    a.n_items = (int32_t)n_items;
    a.err = err;
    a.jobs = jobs;
    a.n_jobs = n_jobs;
    const int64_t clusters = n_items < num_sms / 2 ? n_items : num_sms / 2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * clusters), 1, 1);
    cfg.blockDim = dim3(kPThreads, 1, 1);
    cfg.dynamicSmemBytes = kPSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, correlate_pair_kernel<true, false>, unused, a);
}

}  // namespace xeng
