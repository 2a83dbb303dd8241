// correlate_small.cu -- the whole X-engine step for up to 256 inputs in one
// kernel: the nibble split (paper Sec. II-A) fused into the Hermitian
// correlation (Sec. IV-C-1, Eq. 1), with no decoded planes in HBM, and only
// the upper-triangle 128 x 128 blocks of each channel computed.
//
// A channel of 129..256 inputs has three upper-triangle blocks of 128 inputs:
// (0,0), (0,1) and (1,1).  A pair of CTAs computing the full 256 x 256 product
// does a fourth, (1,0), that the triangle never stores: the two CTAs of a
// cta_group::2 MMA share its B operand, so neither can leave its lower block
// out.  Here each CTA works alone (cta_group::1, M = 128) on items of equal
// cost, each two 128 x 128 complex blocks, 512 TMEM columns:
//   row item of channel c:        A = inputs 0..127, B = inputs 0..255 (one
//                                 N = 256 MMA per product): blocks (0,0), (0,1)
//   diagonal item of channels c, c':  block (1,1) of each (one N = 256 and
//                                 two N = 128 MMAs per product pair)
// Up to 128 inputs a channel is one diagonal block, and every item is a
// diagonal item over two channels' inputs 0..127.  Per stage an item reads two
// raw tiles of 128 inputs x 128 samples ("X" and "Y": the channel's two input
// halves, or the two channels' upper halves).
//
// The launch's work -- its items in order, each of n_k stages of 128 samples --
// is split evenly over the CTAs: CTA b takes stages [b T / G, (b + 1) T / G)
// of that sequence (T stages in all, G CTAs), so every CTA does the same
// number of MMAs whether or not the items divide evenly.  An item cut between
// CTAs is finished by its owner, the CTA holding its first stages (which
// reaches them last): the CTAs holding its later pieces (which start with
// them) write their corrected partial blocks to a workspace and raise a flag
// stamped with the launch's epoch; the owner waits for those flags (bounded),
// adds the partials to its own and stores.  A cooperative launch keeps every
// CTA resident, so the waits end.
//
// The TMA writes raw tiles with a 128-byte swizzle: rows are samples, each 128
// input bytes -- the canonical MN-major layout of an 8-bit tcgen05 operand
// (inputs along M or N, samples along K).  The converter warps split each byte
// at its own offset into the Re plane (high nibble) and the Im plane (low
// nibble) of a plane stage; the raw slots form their own ring, so the TMA runs
// ahead of the conversion.  The MMAs of a row item's stage
// (both operands MN-major; B spans the X and Y tiles, the leading byte offset
// stepping from one to the other):
//     Re += A_re B_re^T + A_im B_im^T,   Im += A_im B_re^T + (-A_re) B_im^T;
// a diagonal item's tile against itself: [B_im | B_re] as one N = 256 operand.
//
// The planes hold raw nibbles: a byte whose low four bits are u (0..15) and
// whose high four bits are clear is the FP8 E4M3 code of u / 512 (the
// subnormal binade and the first normal one share the spacing 2^-9).  With p,
// q the Re and Im nibbles and x = (p - 8) + i (q - 8), over a launch of n
// samples
//     Re V_ij = sum(p_i p_j + q_i q_j) - 8 (S_i + S_j) + 128 n,
//     Im V_ij = sum(q_i p_j - p_i q_j) + 8 (D_i - D_j),
// with S = P + Q, D = P - Q and P, Q the sums of an input's nibbles, which the
// converters form as they split (byte lanes, widened to 16-bit lanes every
// four stages, totalled per piece in shared memory); a piece of an item is
// corrected with its own n and sums, and the pieces' results add up to the
// item's.  The MMA sums are integers / 2^18 of at most 450 n; launches of at
// most 32,768 samples keep them below 2^24, exact in f32.
//
// Roles (576 threads):
//   warp 0       TMA producer: raw tiles into the raw ring
//   warp 1       TMEM allocation; MMA issuer
//   warps 2..9   converters: raw slot -> Re and Im planes of a plane stage, nibble sums
//   warps 10..17 epilogue: TMEM -> packed int32 triangle, one warp per TMEM lane
//                quadrant and block of the item
#include <cstring>

#include "tc_ptx.cuh"
#include "triangle_store.cuh"
#include "xeng_internal.h"

namespace xeng {
namespace {

// Samples per stage (a build parameter, 64 or 128): every stage carries a fixed
// cost in the pipeline (barrier round trips, a commit, the converters' fence),
// so fewer, larger stages run faster although the rings then hold two plane
// stages instead of four (measured on GB300, full Pathfinder rate: 64 samples
// 3.17 ms, 128 samples 2.99 ms).  The rings hold 208 KB (64) or 192 KB (128).
#ifndef XENG_SMALL_KC
#define XENG_SMALL_KC 128
#endif
constexpr int kSKc = XENG_SMALL_KC;         // samples per stage
static_assert(kSKc == 64 || kSKc == 128, "64 or 128 samples per stage");
constexpr int kSBox = kSKc * 128;           // one raw tile or plane tile: kSKc samples x 128 inputs
constexpr int kSRawBytes = 2 * kSBox;       // raw slot: tiles X and Y
constexpr int kSPlaneBytes = 4 * kSBox;     // plane stage: Im_X, Im_Y, Re_X, Re_Y
// Ring depths (build parameters; 4 x 32 KB + 5 x 16 KB fill the shared memory).
#ifndef XENG_SMALL_PLANE_STAGES
#define XENG_SMALL_PLANE_STAGES (4 * 64 / XENG_SMALL_KC)
#endif
#ifndef XENG_SMALL_RAW_SLOTS
#define XENG_SMALL_RAW_SLOTS (XENG_SMALL_KC == 128 ? 2 : 5)
#endif
constexpr int kSPlanes = XENG_SMALL_PLANE_STAGES, kSRaws = XENG_SMALL_RAW_SLOTS;

constexpr int kSConvWarp0 = 2, kSConvWarps = 8;
constexpr int kSEpiWarp0 = kSConvWarp0 + kSConvWarps, kSEpiWarps = 8;
constexpr int kSThreads = 32 * (kSEpiWarp0 + kSEpiWarps);
constexpr uint32_t kSTmemCols = 512;
constexpr int kSSums = 2 * 256 * 8;  // per item parity: (P, Q) of the item's 256 inputs (X tile, then Y tile)
// barriers: raw full and empty per slot, plane full and empty per stage; acc full,
// acc empty, drain; sums full and empty per parity
constexpr int kSBars = 2 * kSRaws + 2 * kSPlanes + 3 + 4;
constexpr size_t kSSmem =
    1024 + (size_t)kSPlanes * kSPlaneBytes + (size_t)kSRaws * kSRawBytes + kSSums + kSBars * 8 + 16;
static_assert(kSSmem <= 232448, "shared memory over the per-CTA limit");
constexpr int kSMinPiece = 32;  // stages per CTA at least (the grid shrinks for small launches)
constexpr int kSChunks = 2 * kSBox / 16 / (32 * kSConvWarps);  // 16-byte chunks per converter thread and stage
static_assert(kSChunks * 32 * kSConvWarps * 16 == 2 * kSBox, "the converter threads cover both tiles");
constexpr int kSWiden = 16 / kSChunks;  // stages between widenings of the byte-lane sums (<= 240)

// Instruction descriptor, kind::f8f6f4: D f32, A and B E4M3, both MN-major
// (bits 15, 16), N = n, M = 128; bit 13 negates A.
__host__ __device__ constexpr uint32_t small_idesc(int n, bool neg_a)
{
    return (1u << 4) | (neg_a ? (1u << 13) : 0u) | (1u << 15) | (1u << 16) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

// MN-major operand with a 128-byte swizzle: rows of 128 elements along M/N,
// 8-row groups along K 1 KB apart (stride byte offset), version 1.  The
// leading byte offset `lbo` is the step between 128-element atoms along M/N,
// where an N = 256 operand continues (one-atom operands ignore it).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

struct SmallArgs {
    int64_t t0, nt;        // samples t0 .. t0 + nt - 1 of the block, nt <= kFusedMaxSamples
    int32_t F, N, f0, nf;  // channels f0 .. f0 + nf - 1
    int32_t n_items, n_k;  // items; stages (of kSKc samples) per item
    int64_t total;         // n_items * n_k: the launch's (item, stage) sequence, split evenly over the CTAs
    int32_t *acc;          // [nf][N(N+1)/2][2], channel f0 + fl at fl
    int accumulate;        // 0: store, 1: add
    int2 *ws;              // [grid][2][16][128][8] partial blocks of pieces that do not start their item
    int *flags;            // [grid]: this launch's epoch once the CTA's partial is in ws
    int *epoch;            // [0]: launches so far on these flags (this launch's epoch is [0] + 1);
                           // [1]: CTAs of this launch finished
    int *err;
    const CUtensorMap *maps;  // null: raw_map over one block; else a map per block of spb stages,
    int32_t spb;              // the launch's samples running through the blocks in order
};

// A CTA's work: the stages [lo, hi) of the launch's sequence (item-major),
// lo = b * total / grid, as pieces (item, stages k0 .. k1 - 1).  A piece with
// k0 > 0 (only ever a CTA's first) adds its partial block through ws; the CTA
// whose piece starts the item (its owner) adds them into its own and stores.
struct Piece {
    int it, k0, k1;
};

__device__ __forceinline__ int64_t range_lo(const SmallArgs &a, int b) { return (int64_t)b * a.total / gridDim.x; }

// The CTA whose range holds stage x of the sequence.
__device__ __forceinline__ int stage_cta(const SmallArgs &a, int64_t x)
{
    return (int)(((x + 1) * (int64_t)gridDim.x - 1) / a.total);
}

__device__ __forceinline__ bool next_piece(const SmallArgs &a, int64_t &x, int64_t hi, Piece &p)
{
    if (x >= hi) return false;
    p.it = (int)(x / a.n_k);
    const int64_t first = (int64_t)p.it * a.n_k;
    p.k0 = (int)(x - first);
    p.k1 = (int)(hi - first < a.n_k ? hi - first : a.n_k);
    x = first + p.k1;
    return true;
}

// Item `it`.  N > 128: per channel pair (2m, 2m + 1) the row item of 2m, the
// diagonal item of both, the row item of 2m + 1 (an odd last channel: its row
// item and a diagonal item of it alone).  N <= 128: diagonal items of channel
// pairs.  fy < 0: no second channel (its tile repeats the first; nothing stored).
struct SmallItem {
    bool row;
    int fx, fy;  // channels (local) of the X and Y tiles
    int base;    // first input of both tiles (diagonal items) / of X (row items: Y at 128)
};

__device__ __forceinline__ SmallItem small_item(const SmallArgs &a, int it)
{
    SmallItem w;
    if (a.N > 128) {
        const int m = it / 3, r = it - 3 * m;
        w.row = r != 1;
        if (w.row) {
            w.fx = w.fy = 2 * m + (r >> 1);
            w.base = 0;
        } else {
            w.fx = 2 * m;
            w.fy = 2 * m + 1 < a.nf ? 2 * m + 1 : -1;
            w.base = 128;
        }
    } else {
        w.row = false;
        w.fx = 2 * it;
        w.fy = 2 * it + 1 < a.nf ? 2 * it + 1 : -1;
        w.base = 0;
    }
    return w;
}

// kAdd: add into acc (a.accumulate != 0) instead of storing; a template so that
// each launch carries only its own triangle-store path (the adding one needs
// more registers).
template <bool kAdd>
__global__ void __launch_bounds__(kSThreads, 1)
correlate_small_kernel(const __grid_constant__ CUtensorMap raw_map, const SmallArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t *sgen = smem_raw + (sbase - raw);
    // plane stages first, then the raw slots, the item sums and the barriers
    const uint32_t raw0 = sbase + kSPlanes * kSPlaneBytes;
    const uint32_t sums_u = raw0 + kSRaws * kSRawBytes;
    const uint32_t bars = sums_u + kSSums;
    int2 *sums = reinterpret_cast<int2 *>(sgen + (sums_u - sbase));  // [parity][256] (P, Q)
    auto plane = [&](int s) { return sbase + (uint32_t)(s * kSPlaneBytes); };
    auto slot = [&](int s) { return raw0 + (uint32_t)(s * kSRawBytes); };
    auto rawf = [&](int s) { return bars + 8u * s; };
    auto rawe = [&](int s) { return bars + 8u * (kSRaws + s); };
    auto full = [&](int s) { return bars + 8u * (2 * kSRaws + s); };
    auto empty = [&](int s) { return bars + 8u * (2 * kSRaws + kSPlanes + s); };
    const uint32_t accf = bars + 8u * (2 * kSRaws + 2 * kSPlanes);
    const uint32_t acce = accf + 8u;
    const uint32_t drain = accf + 16u;
    auto sums_full = [&](int par) { return accf + 24u + 8u * par; };
    auto sums_empty = [&](int par) { return accf + 40u + 8u * par; };
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem_raw + (bars + 8u * kSBars - raw));
    // this launch's flag value, read once at the start: the last CTA of the launch
    // to finish advances the count (at the end), after every CTA has read it here
    int *s_epoch = reinterpret_cast<int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *err = a.err;
    const int64_t lo = range_lo(a, (int)blockIdx.x), hi = range_lo(a, (int)blockIdx.x + 1);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kSRaws; s++) {
            mbar_init(rawf(s), 1);
            mbar_init(rawe(s), kSConvWarps);  // one arrival per converter warp
        }
        for (int s = 0; s < kSPlanes; s++) {
            mbar_init(full(s), kSConvWarps);
            mbar_init(empty(s), 1);
        }
        mbar_init(accf, 1);
        mbar_init(acce, kSEpiWarps);
        mbar_init(drain, 1);
        for (int par = 0; par < 2; par++) {
            mbar_init(sums_full(par), kSConvWarps);
            mbar_init(sums_empty(par), kSEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&raw_map) : "memory");
        *s_epoch = *(volatile int *)a.epoch + 1;
    }
    for (int k = threadIdx.x; k < 2 * 256; k += kSThreads) sums[k] = make_int2(0, 0);
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kSTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int s = 0, issued = 0;
            uint32_t ph = 0;
            bool ok = true;
            int64_t x = lo;
            Piece pc;
            while (ok && next_piece(a, x, hi, pc)) {
                const SmallItem w = small_item(a, pc.it);
                const int fX = a.f0 + w.fx, fY = a.f0 + (w.fy >= 0 ? w.fy : w.fx);
                const int xX = w.base, xY = w.row ? 128 : w.base;
                for (int kc = pc.k0; kc < pc.k1; kc++) {
                    if (!mbar_try_wait(rawe(s), ph ^ 1u) && !mbar_wait(rawe(s), ph ^ 1u, err, kDevTimeoutProducer)) {
                        ok = false;
                        break;
                    }
                    const CUtensorMap *mp = &raw_map;
                    int z = (int)(a.t0 + (int64_t)kc * kSKc);
                    if (a.maps) {  // blocks of spb stages, each with its own map
                        mp = a.maps + kc / a.spb;
                        z = (kc % a.spb) * kSKc;
                    }
                    mbar_expect_tx(rawf(s), kSRawBytes);
                    tma_load_3d(slot(s), mp, xX, fX, z, rawf(s));
                    tma_load_3d(slot(s) + kSBox, mp, xY, fY, z, rawf(s));
                    ++issued;
                    if (++s == kSRaws) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (!ok) {
                // Let the copies already issued land before the CTA can exit.
                for (int k = 1; k <= kSRaws && k <= issued; k++) {
                    int sk = s - k, p = (int)ph;
                    if (sk < 0) { sk += kSRaws; p ^= 1; }
                    (void)mbar_wait(rawf(sk), (uint32_t)p, err, kDevTimeoutProducer);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            int s = 0;
            uint32_t ph = 0, uses = 0;
            bool ok = true;
            int64_t x = lo;
            Piece pc;
            while (ok && next_piece(a, x, hi, pc)) {
                const SmallItem w = small_item(a, pc.it);
                if (!mbar_wait(acce, (uses & 1u) ^ 1u, err, kDevTimeoutMma)) break;
                ++uses;
                fence_after();
                for (int kc = pc.k0; kc < pc.k1; kc++) {
                    if (!mbar_try_wait(full(s), ph) && !mbar_wait(full(s), ph, err, kDevTimeoutMma)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t st = plane(s);
                    if (w.row) {
                        // A = X rows, B = X and Y columns (the Y plane kSBox after the X
                        // plane): Re in columns 0..255, Im in 256..511
                        const uint64_t dre = sdesc(st + 2 * kSBox, kSBox), dim = sdesc(st, kSBox);
                        #pragma unroll
                        for (int kk = 0; kk < kSKc / 32; kk++) {  // +32 samples = +4 KB = +256 in the address field
                            const uint32_t acc = (kc != pc.k0 || kk != 0) ? 1u : 0u;
                            const uint64_t k4 = 256u * kk;
                            mma_f8(tmem, dre + k4, dre + k4, small_idesc(256, false), acc);
                            mma_f8(tmem, dim + k4, dim + k4, small_idesc(256, false), 1u);
                            mma_f8(tmem + 256u, dim + k4, dre + k4, small_idesc(256, false), acc);
                            mma_f8(tmem + 256u, dre + k4, dim + k4, small_idesc(256, true), 1u);
                        }
                    } else {
                        // each tile against itself, in columns 256h..: one N = 256 MMA of
                        // A_im against [B_im | B_re] (Re_h 16 KB after Im_h) gives
                        // [Im Im^T | Im Re^T]; A_re B_re^T completes Re, and (-A_re) B_im^T
                        // makes the second half Im Re^T - Re Im^T = Im.  (Four N = 128 MMAs
                        // per tile instead ran at about 72% of the tensor rate.)
                        #pragma unroll
                        for (int h = 0; h < 2; h++) {
                            const uint64_t dim = sdesc(st + h * kSBox, 2 * kSBox), dre = sdesc(st + (2 + h) * kSBox, 2 * kSBox);
                            const uint32_t d = tmem + 256u * h;
                            #pragma unroll
                            for (int kk = 0; kk < kSKc / 32; kk++) {
                                const uint32_t acc = (kc != pc.k0 || kk != 0) ? 1u : 0u;
                                const uint64_t k4 = 256u * kk;
                                mma_f8(d, dim + k4, dim + k4, small_idesc(256, false), acc);
                                mma_f8(d, dre + k4, dre + k4, small_idesc(128, false), 1u);
                                mma_f8(d + 128u, dre + k4, dim + k4, small_idesc(128, true), 1u);
                            }
                        }
                    }
                    mma_commit(empty(s));
                    if (++s == kSPlanes) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit(accf);
            }
            // Drain: every MMA issued above has finished once this completes.
            mma_commit(drain);
            (void)mbar_wait(drain, 0u, err, kDevTimeoutMma);
        }
    } else if (warp < kSEpiWarp0) {
        // ---------------- converters ----------------
        // Thread u (0..255) takes tile g = u / 128 and, in it, the 16-byte chunks
        // v + 128 k (v = u % 128, k < kSChunks): sample rows v / 8 + 16 k,
        // physical chunk v % 8 -- a quarter-warp covers one whole 128-byte row, so
        // the accesses are bank-conflict-free.  The rows' swizzle (chunk ^ row % 8)
        // is the same for all of them, so the thread always holds the same 16
        // inputs: logical chunk lc = (v % 8) ^ (v / 8 % 8).
        const int u = (warp - kSConvWarp0) * 32 + lane;
        const int g = u >> 7, v = u & 127;
        const int r0 = v >> 3, lc = (v & 7) ^ (r0 & 7);
        const uint32_t off0 = (uint32_t)(g * kSBox + v * 16);  // chunk k at off0 + 2048 k within a slot / plane pair
        const int nt = (int)a.nt;                               // <= kFusedMaxSamples
        int rs = 0, ps = 0, local = 0;
        uint32_t rph = 0, pph = 0;
        bool ok = true;
        int64_t x = lo;
        Piece pc;
        for (; ok && next_piece(a, x, hi, pc); ++local) {
            // nibble sums of the thread's 16 inputs: byte lanes over up to 16
            // samples (<= 240), then 16-bit lanes (<= 15 x 2048 samples)
            uint32_t pb[4] = {0, 0, 0, 0}, qb[4] = {0, 0, 0, 0};
            uint32_t P16[8] = {0, 0, 0, 0, 0, 0, 0, 0}, Q16[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            auto widen = [&]() {
                #pragma unroll
                for (int w = 0; w < 4; w++) {
                    P16[2 * w] += pb[w] & 0x00FF00FFu;
                    P16[2 * w + 1] += (pb[w] >> 8) & 0x00FF00FFu;
                    Q16[2 * w] += qb[w] & 0x00FF00FFu;
                    Q16[2 * w + 1] += (qb[w] >> 8) & 0x00FF00FFu;
                    pb[w] = qb[w] = 0;
                }
            };
            for (int kc = pc.k0; kc < pc.k1; kc++) {
                ok = mbar_wait_backoff(rawf(rs), rph, err, kDevTimeoutProducer, XENG_CONV_SLEEP_NS);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                const int rows_left = nt - kc * kSKc;  // samples of this stage inside the launch (may exceed kSKc)
                const uint8_t *src = sgen + (slot(rs) - sbase) + off0;
                uint4 x[kSChunks];
                #pragma unroll
                for (int k = 0; k < kSChunks; k++) {
                    x[k] = *reinterpret_cast<const uint4 *>(src + 2048 * k);
                    if (r0 + 16 * k >= rows_left) x[k] = make_uint4(0, 0, 0, 0);  // past the launch: adds nothing
                }
                // The raw slot goes back to the producer with the plane stage below, once
                // the plane stores (which consume the loaded words) are done.  An arrival
                // right after the loads, with nothing waiting for their data, let the TMA
                // refill the slot under loads still in flight (measured on GB300: whole
                // items wrong in about one launch in two when the MMAs stalled behind a
                // long epilogue); one whose address depended on the loaded words was
                // exact but 1% slower than this.
                const int rcur = rs;
                if (++rs == kSRaws) {
                    rs = 0;
                    rph ^= 1u;
                }
                ok = mbar_wait_backoff(empty(ps), pph ^ 1u, err, kDevTimeoutProducer, XENG_CONV_SLEEP_NS);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                uint8_t *dim = sgen + (plane(ps) - sbase) + off0;  // Im_X / Im_Y
                uint8_t *dre = dim + 2 * kSBox;                    // Re_X / Re_Y
                #pragma unroll
                for (int k = 0; k < kSChunks; k++) {
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
                    mbar_arrive(full(ps));
                    mbar_arrive(rawe(rcur));
                }
                if (++ps == kSPlanes) {
                    ps = 0;
                    pph ^= 1u;
                }
                if ((kc - pc.k0 + 1) % kSWiden == 0) widen();
            }
            if (!ok) break;
            widen();
            // the four lanes of a warp holding the same inputs (rows differing in
            // their two low bits: lanes ^ 9, ^ 18) add up -- two in 16-bit lanes
            // (<= 2 x 15 x 2048), the other two in 32 bits -- then one of them adds
            // the warp's totals into the item's sums; input 4w + b is byte b of word w
            uint32_t P32[16], Q32[16];
            #pragma unroll
            for (int k = 0; k < 8; k++) {
                P16[k] += __shfl_xor_sync(0xffffffffu, P16[k], 9);
                Q16[k] += __shfl_xor_sync(0xffffffffu, Q16[k], 9);
            }
            #pragma unroll
            for (int m = 0; m < 16; m++) {
                const int w = m >> 2, b = m & 3;
                P32[m] = (P16[2 * w + (b & 1)] >> (16 * (b >> 1))) & 0xFFFFu;
                Q32[m] = (Q16[2 * w + (b & 1)] >> (16 * (b >> 1))) & 0xFFFFu;
                P32[m] += __shfl_xor_sync(0xffffffffu, P32[m], 18);
                Q32[m] += __shfl_xor_sync(0xffffffffu, Q32[m], 18);
            }
            const int par = local & 1;
            // the buffer was last read (and cleared) by the epilogue two items ago
            ok = mbar_wait_backoff(sums_empty(par), (uint32_t)((local >> 1) & 1) ^ 1u, err, kDevTimeoutProducer,
                                   XENG_CONV_SLEEP_NS);
            if (!__all_sync(0xffffffffu, ok)) {
                ok = false;
                break;
            }
            if ((r0 & 3) == 0) {
                int *sp = reinterpret_cast<int *>(sums + par * 256 + g * 128 + lc * 16);
                #pragma unroll
                for (int m = 0; m < 16; m++) {
                    atomicAdd(sp + 2 * m, (int)P32[m]);
                    atomicAdd(sp + 2 * m + 1, (int)Q32[m]);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(sums_full(par));
        }
    } else {
        // ---------------- epilogue ----------------
        const int q = warp & 3;                     // TMEM lane quadrant this warp may access
        const int h = (warp - kSEpiWarp0) >> 2;     // the item's block: columns 128h.. of Re and Im
        const int et = (warp - kSEpiWarp0) * 32 + lane;
        const int row = q * 32 + lane;              // TMEM lane: row within the block
        const int N = a.N;                          // <= 256
        const int nt = (int)a.nt;
        const int64_t nb = (int64_t)N * (N + 1) / 2;
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16);
        // partial blocks in ws: [CTA][block h][chunk c / 8][row][8 pairs]
        constexpr int kWs = 2 * 16 * 128 * 8;
        const int wsi = ((h * 16) * 128 + row) * 8;  // + (c / 8) * 1024
        uint32_t uses = 0;
        int local = 0;
        int64_t x = lo;
        Piece pc;
        while (next_piece(a, x, hi, pc)) {
            const SmallItem w = small_item(a, pc.it);
            const int par = local & 1;
            // the piece's samples inside the launch: 64 n from each of the two products
            const int n128 = 128 * ((pc.k1 * kSKc < nt ? pc.k1 * kSKc : nt) - pc.k0 * kSKc);
            const bool owner = pc.k0 == 0;
            // an owner whose item runs on: the CTAs after it that hold the rest
            const int c_lo = (int)blockIdx.x + 1;
            const int c_hi = owner && pc.k1 < a.n_k ? stage_cta(a, (int64_t)(pc.it + 1) * a.n_k - 1) : 0;
            bool ok = mbar_wait_backoff(accf, uses & 1u, err, kDevTimeoutEpilogue, 128);
            ok = ok && mbar_wait_backoff(sums_full(par), (uint32_t)((local >> 1) & 1), err, kDevTimeoutEpilogue, 128);
            if (et == 0)
                for (int b = c_lo; ok && b <= c_hi; b++) ok = flag_wait(a.flags + b, *s_epoch, err, kDevTimeoutEpilogue);
            // the barrier ORs the eight warps' failures, so they leave together
            if (bar_any(2, kSEpiWarps * 32, !ok)) break;
            ++uses;
            fence_after();
            // block geometry: row items (rows 0..127, columns 128h..), diagonal items
            // (channel fx or fy, rows and columns base..); sums index: X tile 0..127, Y tile 128..
            const int fl = w.row ? w.fx : (h ? w.fy : w.fx);
            const int i0 = w.row ? 0 : w.base;
            const int j0b = w.row ? 128 * h : w.base;
            const int2 *srow = sums + par * 256 + (w.row ? 0 : 128 * h);
            const int2 *scol = sums + par * 256 + 128 * h;
            const int i_warp = i0 + q * 32;
            const int i = i0 + row;
            if (fl >= 0 && i_warp < N) {
                const bool row_ok = i < N;
                const int2 pq = srow[row];
                const int si = pq.x + pq.y, di = pq.x - pq.y;
                const int row_base = i * N - i * (i - 1) / 2 - i;  // pair (i, j) at row_base + j
                int2 *out = reinterpret_cast<int2 *>(a.acc) + (int64_t)fl * nb;
                // TMEM columns of the block: row items Re at 128h.., Im at 256 + 128h..;
                // diagonal items Re at 256h.., Im at 256h + 128..
                const uint32_t cre = w.row ? 128u * h : 256u * h;
                const uint32_t cim = cre + (w.row ? 256u : 128u);
                for (int c = 0; c < 128; c += 8) {
                    const int j0 = j0b + c;
                    // warp-uniform skips: chunks past the last input or below every row's diagonal
                    if (j0 >= N) break;
                    if (j0 + 7 < i_warp) continue;
                    uint32_t vre[8], vim[8];
                    tmem_ld8(taddr + cre + c, vre);
                    tmem_ld8(taddr + cim + c, vim);
                    tmem_ld_wait();
                    if (!row_ok) continue;
                    #pragma unroll
                    for (int e = 0; e < 8; e++) {  // corrected values in place of the accumulator words
                        const int2 pj = scol[c + e];  // the same for every lane: a broadcast
                        // accumulators hold integer sums / 2^18: x 2^18 is exact
                        vre[e] = (uint32_t)(__float2int_rn(262144.0f * __uint_as_float(vre[e])) -
                                            8 * (si + pj.x + pj.y) + n128);
                        vim[e] = (uint32_t)(__float2int_rn(262144.0f * __uint_as_float(vim[e])) +
                                            8 * (di - (pj.x - pj.y)));
                    }
                    const int wo = wsi + (c >> 3) * 1024;
                    if (!owner) {
                        // a later piece of the item: the partial goes to this CTA's slot
                        int4 *d = reinterpret_cast<int4 *>(a.ws + (int64_t)blockIdx.x * kWs + wo);
                        #pragma unroll
                        for (int e = 0; e < 8; e += 2)
                            __stcg(d + e / 2, make_int4((int)vre[e], (int)vim[e], (int)vre[e + 1], (int)vim[e + 1]));
                        continue;
                    }
                    for (int b = c_lo; b <= c_hi; b++) {  // the item's later pieces (none for a whole item)
                        const int4 *src = reinterpret_cast<const int4 *>(a.ws + (int64_t)b * kWs + wo);
                        #pragma unroll
                        for (int e = 0; e < 8; e += 2) {
                            const int4 v = __ldcg(src + e / 2);
                            vre[e] += (uint32_t)v.x;
                            vim[e] += (uint32_t)v.y;
                            vre[e + 1] += (uint32_t)v.z;
                            vim[e + 1] += (uint32_t)v.w;
                        }
                    }
                    put8<kAdd>(out + row_base + j0, i - j0, N - j0, vre, vim);
                }
            }
            if (!owner) __threadfence();  // the partial is visible at GPU scope before the flag below
            // every epilogue thread is done with this parity's sums: clear them for
            // the piece after next, then hand TMEM and the buffer back
            named_bar_sync(2, kSEpiWarps * 32);
            if (!owner && et == 0) st_release_gpu(a.flags + blockIdx.x, *s_epoch);
            sums[par * 256 + et] = make_int2(0, 0);
            fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(acce);
                mbar_arrive(sums_empty(par));
            }
            ++local;
        }
    }

    __syncwarp();
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kSTmemCols));
    }
    // One launch more on these flags: the last CTA to get here (every CTA read the
    // epoch when it started, before getting here) advances the count and resets
    // the arrivals, so the next launch -- or the next replay of a captured one --
    // takes a fresh epoch.  Epochs run 1 .. 2^31 - 1, never 0 (an unset flag).
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.epoch + 1, 1) == (int)gridDim.x - 1) {
            const int e = *(volatile int *)a.epoch;
            a.epoch[1] = 0;
            a.epoch[0] = e >= 0x7FFFFFFE ? 0 : e + 1;
            __threadfence();
        }
    }
}

}  // namespace

bool small_ok(const uint8_t *block, int32_t N)
{
    return N >= 1 && N <= 256 && N % 16 == 0 && (reinterpret_cast<uintptr_t>(block) & 15) == 0;
}

size_t small_ws_bytes(int num_sms) { return (size_t)num_sms * 2 * 16 * 128 * 8 * sizeof(int2); }
size_t small_flags_bytes(int num_sms) { return (size_t)(num_sms + 2) * sizeof(int); }

cudaError_t encode_small_map(CUtensorMap *map, const uint8_t *block, int64_t T_block, int32_t F, int32_t N)
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    // raw block: dims (input, channel, sample), boxes of 128 inputs x 1 channel x kSKc
    // samples with a 128-byte swizzle (the MN-major operand layout); inputs past N and
    // samples past the block read as zero bytes, nibbles 0 that add nothing (the
    // converters zero the samples past the launch; rows and columns past N are never
    // written)
    cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)F, (cuuint64_t)T_block};
    cuuint64_t strides[2] = {(cuuint64_t)N, (cuuint64_t)N * F};
    cuuint32_t box[3] = {128, 1, (cuuint32_t)kSKc}, estr[3] = {1, 1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, (void *)block, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

int small_stage_samples() { return kSKc; }

cudaError_t launch_correlate_small(const uint8_t *block, int64_t T_block, int64_t t0, int64_t nt, int32_t F, int32_t N,
                                   int32_t f0, int32_t nf, int32_t *acc, int accumulate, int2 *ws, int *flags,
                                   int *err, int num_sms, cudaStream_t s,
                                   const CUtensorMap *maps, int32_t spb)
{
    if (nf <= 0 || nt <= 0) return cudaSuccess;
    if (!small_ok(maps ? nullptr : block, N) || (maps && (spb < 1 || t0 != 0)) || nt > kFusedMaxSamples ||
        t0 < 0 || t0 + nt > T_block || T_block > 2147483647LL ||
        f0 < 0 || f0 + nf > F || num_sms < 1 || (reinterpret_cast<uintptr_t>(acc) & 7) != 0 || !ws || !flags)
        return cudaErrorInvalidValue;
    const int64_t n_items = N > 128 ? (int64_t)nf + (nf + 1) / 2 : (int64_t)(nf + 1) / 2;
    const int n_k = (int)((nt + kSKc - 1) / kSKc);
    CUtensorMap map;
    if (maps) {
        memset(&map, 0, sizeof map);  // not read: the stages take the blocks' maps
    } else {
        cudaError_t e0 = encode_small_map(&map, block, T_block, F, N);
        if (e0 != cudaSuccess) return e0;
    }
    auto kern = accumulate ? correlate_small_kernel<true> : correlate_small_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSSmem);
    if (e != cudaSuccess) return e;
    SmallArgs a;
    a.t0 = t0;
    a.nt = nt;
    a.F = F;
    a.N = N;
    a.f0 = f0;
    a.nf = nf;
    a.n_items = (int32_t)n_items;
    a.n_k = n_k;
    a.total = n_items * n_k;
    a.acc = acc;
    a.accumulate = accumulate;
    a.ws = ws;
    a.flags = flags;
    a.epoch = flags + num_sms;
    a.err = err;
    a.maps = maps;
    a.spb = spb;
    // every CTA gets at least kSMinPiece stages (a piece's epilogue and partial
    // cost about as much as a few stages of MMAs), at most one CTA per SM
    int64_t grid = a.total / kSMinPiece;
    if (grid < 1) grid = 1;
    if (grid > num_sms) grid = num_sms;
    // the owner of a split item waits for the CTAs holding its later pieces:
    // a cooperative launch has every CTA resident at once (or fails)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(kSThreads, 1, 1);
    cfg.dynamicSmemBytes = kSSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, map, a);
}

}  // namespace xeng
