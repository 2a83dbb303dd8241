// correlate_onepass.cu -- the X-engine step in one pass over the raw bytes
// with single CTAs over 128-input block pairs: the nibble split (paper Sec.
// II-A) fused into the Hermitian correlation (Sec. IV-C-1, Eq. 1), with no
// decoded planes in HBM.
//
// A separate decode writes two plane bytes per input byte to HBM and the
// correlation reads them back.  Converting in shared memory instead takes the
// converter warps' time: each 128 x 128 block pair converts two raw tiles per
// 1024 MMA cycles (per 128-sample stage), so this kernel runs
// at about 60% of the MMA rate -- ahead of the two passes while the decode is a
// large share of the step; the library runs it for N > 256 where ceil(N / 128)
// is odd (there the 2-CTA kernel over 256-input block pairs pads N the most).
// Each CTA (one per SM, cta_group::1) takes upper-triangle tile pairs (I <= J)
// of 128-input blocks of a channel, channel-major and round-robin over the
// CTAs, so the CTAs at work at any time share one or two channels' raw bytes in
// L2.  Per stage of kOKc samples the producer TMA-loads the raw bytes of block
// J (the A operand: TMEM lanes are inputs j) and block I (B: columns are inputs
// i; only one tile on the diagonal) with a 128-byte swizzle -- the canonical
// MN-major layout of an 8-bit tcgen05 operand -- into a raw ring; converter
// warps split each byte at its own offset into the Im and Re planes of a plane
// stage and sum each input's nibbles.  Per 32-sample K step the MMA thread
// issues
//     D[:, 0:256]   = A_im x [B_im | B_re]^T   (N = 256; B_re after B_im)
//     D[:, 0:128]  += A_re x B_re^T            (N = 128)  -> sum(p_i p_j + q_i q_j)
//     D[:, 128:256]+= (-A_re) x B_im^T         (N = 128)  -> sum(q_j p_i - p_j q_i)
// into one of two 256-column TMEM accumulators, so the epilogue of a tile pair
// overlaps the MMAs of the next; the epilogue negates the Im half (with A = x_j
// it is minus Im of x_i conj(x_j)), and per column i a warp's 32 lanes write
// 32 consecutive pairs of the triangle's row i (one 256-byte run).
//
// The planes hold raw nibbles: a byte whose low four bits are u (0..15) and
// whose high four bits are clear is the FP8 E4M3 code of u / 512.  With p, q
// the Re and Im nibbles and x = (p - 8) + i (q - 8), over a launch of n samples
//     Re V_ij = sum(p_i p_j + q_i q_j) - 8 (S_i + S_j) + 128 n,
//     Im V_ij = sum(q_i p_j - p_i q_j) + 8 (D_i - D_j),
// with S = P + Q, D = P - Q and P, Q the sums of an input's nibbles, which the
// converters form per tile pair as they split.  The MMA sums are integers /
// 2^18 of at most 450 n; launches of at most 32,768 samples keep them below
// 2^24, exact in f32.
//
// Roles (576 threads):
//   warp 0       TMA producer: raw tiles into the raw ring
//   warp 1       TMEM allocation; MMA issuer
//   warps 2..9   converters: raw slot -> Im and Re planes of a plane stage, nibble sums
//   warps 10..17 epilogue: TMEM -> packed int32 triangle, two warps per TMEM lane
//                quadrant taking alternate 8-column chunks
#include <cstring>

#include "tc_ptx.cuh"
#include "xeng_internal.h"

namespace xeng {
namespace {

// Samples per stage (a build parameter: 32, 64 or 128); the rings hold 208 KB
// (32, 64) or 192 KB (128) of stages.  Each stage carries a fixed cost in the
// pipeline: measured on GB300 (N = 512 / 2048, F = 1024, T = 8192) 32 samples
// 5.87 / 81.9 ms, 64 4.32 / 61.0, 128 3.66 / 58.8.
#ifndef XENG_ONEPASS_KC
#define XENG_ONEPASS_KC 128
#endif
constexpr int kOKc = XENG_ONEPASS_KC;       // samples per stage
static_assert(kOKc == 32 || kOKc == 64 || kOKc == 128, "32, 64 or 128 samples per stage");
constexpr int kOBox = kOKc * 128;           // one raw tile or plane tile: kOKc samples x 128 inputs
constexpr int kORawBytes = 2 * kOBox;       // raw slot: blocks I and J
constexpr int kOPlaneBytes = 4 * kOBox;     // plane stage: A_im, A_re, B_im, B_re
// Ring depths (build parameters; 4 x 32 KB + 5 x 16 KB fill the shared memory).
#ifndef XENG_ONEPASS_PLANE_STAGES
#define XENG_ONEPASS_PLANE_STAGES (4 * 64 / XENG_ONEPASS_KC)
#endif
#ifndef XENG_ONEPASS_RAW_SLOTS
#define XENG_ONEPASS_RAW_SLOTS (XENG_ONEPASS_KC == 128 ? 2 : 5 * 64 / XENG_ONEPASS_KC)
#endif
constexpr int kOPlanes = XENG_ONEPASS_PLANE_STAGES, kORaws = XENG_ONEPASS_RAW_SLOTS;
// Converter and epilogue warps (build parameters): the converters' throughput
// bounds the kernel, the epilogue overlaps the next pair's MMAs.
#ifndef XENG_ONEPASS_CONV_WARPS
#define XENG_ONEPASS_CONV_WARPS 8
#endif
#ifndef XENG_ONEPASS_EPI_WARPS
#define XENG_ONEPASS_EPI_WARPS 8
#endif
constexpr int kOConvWarp0 = 2, kOConvWarps = XENG_ONEPASS_CONV_WARPS;
constexpr int kOEpiWarp0 = kOConvWarp0 + kOConvWarps, kOEpiWarps = XENG_ONEPASS_EPI_WARPS;
constexpr int kOThreads = 32 * (kOEpiWarp0 + kOEpiWarps);
constexpr int kOCT = 16 * kOConvWarps;        // converter threads per tile
constexpr int kOChunks = kOBox / 16 / kOCT;   // 16-byte chunks of a tile per converter thread and stage
static_assert(kOConvWarps == 8 || kOConvWarps == 16, "8 or 16 converter warps");
static_assert(kOEpiWarps == 4 || kOEpiWarps == 8, "4 or 8 epilogue warps");
constexpr uint32_t kOTmemCols = 512;
constexpr int kOSums = 2 * 256 * 8;  // per item parity: (P, Q) of block I's inputs, then block J's
// barriers: raw full and empty per slot, plane full and empty per stage; acc full
// and empty per accumulator; drain; sums full and empty per parity
constexpr int kOBars = 2 * kORaws + 2 * kOPlanes + 4 + 1 + 4;
constexpr size_t kOSmem =
    1024 + (size_t)kOPlanes * kOPlaneBytes + (size_t)kORaws * kORawBytes + kOSums + kOBars * 8 + 16;
static_assert(kOSmem <= 232448, "shared memory over the per-CTA limit");
static_assert(kOChunks * kOCT * 16 == kOBox, "the converter threads cover a tile");
constexpr int kOWiden = 16 / kOChunks;        // stages between widenings of the byte-lane sums (<= 240)

// Instruction descriptor, kind::f8f6f4: D f32, A and B E4M3, both MN-major
// (bits 15, 16), N = n, M = 128; bit 13 negates A.
__host__ __device__ constexpr uint32_t op_idesc(int n, bool neg_a)
{
    return (1u << 4) | (neg_a ? (1u << 13) : 0u) | (1u << 15) | (1u << 16) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

// MN-major operand with a 128-byte swizzle: rows of 128 elements along M/N,
// 8-row groups along K 1 KB apart (stride byte offset), version 1; the
// leading byte offset (kOBox) is the step to the second 128-element atom of an
// N = 256 operand: the Re plane after the Im plane of the same block.
__device__ __forceinline__ uint64_t odesc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(kOBox >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

struct OnepassArgs {
    int64_t t0, nt;        // samples t0 .. t0 + nt - 1 of the block, nt <= kFusedMaxSamples
    int32_t F, N, f0, nf;  // channels f0 .. f0 + nf - 1
    int32_t nb;            // 128-input blocks
    int32_t pairs_per_ch;  // nb (nb + 1) / 2
    int32_t n_items;       // nf * pairs_per_ch
    int32_t *acc;          // [nf][N(N+1)/2][2], channel f0 + fl at fl
    int accumulate;        // 0: store, 1: add
    int *err;
    const CUtensorMap *maps;  // null: raw_map over one block; else a map per block of spb stages,
    int32_t spb;              // the launch's samples running through the blocks in order
};

struct OnepassItem {
    int fl, I, J;
};

// Item `it`: channel-major, the channel's block pairs I <= J row by row.
__device__ __forceinline__ OnepassItem onepass_item(const OnepassArgs &a, int it)
{
    OnepassItem w;
    w.fl = it / a.pairs_per_ch;
    int r = it - w.fl * a.pairs_per_ch, i = 0;
    while (r >= a.nb - i) {
        r -= a.nb - i;
        ++i;
    }
    w.I = i;
    w.J = i + r;
    return w;
}

// kAdd: the launch adds to the triangle (a later piece of an integration)
// instead of storing it; a separate instantiation, so the storing epilogue
// keeps two chunks' TMEM words in registers without spilling.
template <bool kAdd>
__global__ void __launch_bounds__(kOThreads, 1)
correlate_onepass_kernel(const __grid_constant__ CUtensorMap raw_map, const OnepassArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t *sgen = smem_raw + (sbase - raw);
    // plane stages first, then the raw slots, the item sums and the barriers
    const uint32_t raw0 = sbase + kOPlanes * kOPlaneBytes;
    const uint32_t sums_u = raw0 + kORaws * kORawBytes;
    const uint32_t bars = sums_u + kOSums;
    int2 *sums = reinterpret_cast<int2 *>(sgen + (sums_u - sbase));  // [parity][256] (P, Q)
    auto plane = [&](int s) { return sbase + (uint32_t)(s * kOPlaneBytes); };
    auto slot = [&](int s) { return raw0 + (uint32_t)(s * kORawBytes); };
    auto rawf = [&](int s) { return bars + 8u * s; };
    auto rawe = [&](int s) { return bars + 8u * (kORaws + s); };
    auto full = [&](int s) { return bars + 8u * (2 * kORaws + s); };
    auto empty = [&](int s) { return bars + 8u * (2 * kORaws + kOPlanes + s); };
    const uint32_t acc0 = bars + 8u * (2 * kORaws + 2 * kOPlanes);
    auto accf = [&](int b) { return acc0 + 8u * b; };
    auto acce = [&](int b) { return acc0 + 16u + 8u * b; };
    const uint32_t drain = acc0 + 32u;
    auto sums_full = [&](int par) { return acc0 + 40u + 8u * par; };
    auto sums_empty = [&](int par) { return acc0 + 56u + 8u * par; };
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem_raw + (bars + 8u * kOBars - raw));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *err = a.err;
    const int it_begin = (int)blockIdx.x, it_step = (int)gridDim.x;
    const int n_k = (int)((a.nt + kOKc - 1) / kOKc);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kORaws; s++) {
            mbar_init(rawf(s), 1);
            mbar_init(rawe(s), kOConvWarps);  // one arrival per converter warp
        }
        for (int s = 0; s < kOPlanes; s++) {
            mbar_init(full(s), kOConvWarps);
            mbar_init(empty(s), 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(accf(b), 1);
            mbar_init(acce(b), kOEpiWarps);
        }
        mbar_init(drain, 1);
        for (int par = 0; par < 2; par++) {
            mbar_init(sums_full(par), kOConvWarps);
            mbar_init(sums_empty(par), kOEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&raw_map) : "memory");
    }
    for (int k = threadIdx.x; k < 2 * 256; k += kOThreads) sums[k] = make_int2(0, 0);
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kOTmemCols));
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
            for (int it = it_begin; ok && it < a.n_items; it += it_step) {
                const OnepassItem w = onepass_item(a, it);
                const int f = a.f0 + w.fl;
                const bool diag = w.I == w.J;
                for (int kc = 0; kc < n_k; kc++) {
                    if (!mbar_try_wait(rawe(s), ph ^ 1u) && !mbar_wait(rawe(s), ph ^ 1u, err, kDevTimeoutProducer)) {
                        ok = false;
                        break;
                    }
                    const CUtensorMap *mp = &raw_map;
                    int z = (int)(a.t0 + (int64_t)kc * kOKc);
                    if (a.maps) {  // blocks of spb stages, each with its own map
                        mp = a.maps + kc / a.spb;
                        z = (kc % a.spb) * kOKc;
                    }
                    mbar_expect_tx(rawf(s), diag ? kOBox : kORawBytes);
                    // A: block J (TMEM lanes = inputs j), B: block I (columns = inputs i)
                    tma_load_3d(slot(s), mp, w.J * 128, f, z, rawf(s));
                    if (!diag) tma_load_3d(slot(s) + kOBox, mp, w.I * 128, f, z, rawf(s));
                    ++issued;
                    if (++s == kORaws) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (!ok) {
                // Let the copies already issued land before the CTA can exit.
                for (int k = 1; k <= kORaws && k <= issued; k++) {
                    int sk = s - k, p = (int)ph;
                    if (sk < 0) { sk += kORaws; p ^= 1; }
                    (void)mbar_wait(rawf(sk), (uint32_t)p, err, kDevTimeoutProducer);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            int local = 0;
            for (int it = it_begin; ok && it < a.n_items; it += it_step, ++local) {
                const OnepassItem w = onepass_item(a, it);
                const bool diag = w.I == w.J;
                // accumulator ab = local % 2, used for the (local / 2)-th time
                const int ab = local & 1;
                if (!mbar_wait(acce(ab), (uint32_t)((local >> 1) & 1) ^ 1u, err, kDevTimeoutMma)) break;
                fence_after();
                const uint32_t d = tmem + 256u * ab;
                for (int kc = 0; kc < n_k; kc++) {
                    if (!mbar_try_wait(full(s), ph) && !mbar_wait(full(s), ph, err, kDevTimeoutMma)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t st = plane(s);
                    // A: block J (Im plane, Re kOBox on); B: block I, or J itself on the diagonal
                    const uint64_t da_im = odesc(st), da_re = odesc(st + kOBox);
                    const uint64_t db_im = diag ? da_im : odesc(st + 2 * kOBox);
                    const uint64_t db_re = diag ? da_re : odesc(st + 3 * kOBox);
                    #pragma unroll
                    for (int kk = 0; kk < kOKc / 32; kk++) {  // +32 samples = +4 KB = +256 in the address field
                        const uint32_t acc = (kc != 0 || kk != 0) ? 1u : 0u;
                        const uint64_t k4 = 256u * kk;
                        mma_f8(d, da_im + k4, db_im + k4, op_idesc(256, false), acc);
                        mma_f8(d, da_re + k4, db_re + k4, op_idesc(128, false), 1u);
                        mma_f8(d + 128u, da_re + k4, db_im + k4, op_idesc(128, true), 1u);
                    }
                    mma_commit(empty(s));
                    if (++s == kOPlanes) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit(accf(ab));
            }
            // Drain: every MMA issued above has finished once this completes.
            mma_commit(drain);
            (void)mbar_wait(drain, 0u, err, kDevTimeoutMma);
        }
    } else if (warp < kOEpiWarp0) {
        // ---------------- converters ----------------
        // Thread u takes tile g = u / kOCT (block I, then J) and, in it, the
        // 16-byte chunks v + kOCT k (v = u % kOCT, k < kOChunks): sample rows
        // v / 8 + kOCT / 8 k, physical chunk v % 8 -- a quarter-warp covers one
        // whole 128-byte row, so the accesses are bank-conflict-free.  The rows'
        // swizzle (chunk ^ row % 8) is the same for all of them (kOCT / 8 is a
        // multiple of 8), so the thread always holds the same 16 inputs: logical
        // chunk lc = (v % 8) ^ (v / 8 % 8).
        const int u = (warp - kOConvWarp0) * 32 + lane;
        const int g = u / kOCT, v = u % kOCT;
        const int r0 = v >> 3, lc = (v & 7) ^ (r0 & 7);
        const uint32_t roff = (uint32_t)(g * kOBox + v * 16);      // in a raw slot (+ 16 kOCT k)
        const uint32_t poff = (uint32_t)(2 * g * kOBox + v * 16);  // Im plane of the tile (+ 16 kOCT k; Re kOBox on)
        const int nt = (int)a.nt;                                  // <= kFusedMaxSamples
        int rs = 0, ps = 0, local = 0;
        uint32_t rph = 0, pph = 0;
        bool ok = true;
        for (int it = it_begin; ok && it < a.n_items; it += it_step, ++local) {
            const OnepassItem w = onepass_item(a, it);
            const bool active = g == 0 || w.I != w.J;  // the diagonal has block I only
            // nibble sums of the thread's 16 inputs: byte lanes over up to four
            // stages (16 samples, <= 240), then 16-bit lanes (<= 15 x 2048 samples)
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
            for (int kc = 0; kc < n_k; kc++) {
                ok = mbar_wait_backoff(rawf(rs), rph, err, kDevTimeoutProducer, XENG_CONV_SLEEP_NS);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                const int rows_left = nt - kc * kOKc;  // samples of this stage inside the launch (may exceed kOKc)
                const uint8_t *src = sgen + (slot(rs) - sbase) + roff;
                uint4 x[kOChunks];
                #pragma unroll
                for (int k = 0; k < kOChunks; k++) {
                    x[k] = active ? *reinterpret_cast<const uint4 *>(src + 16 * kOCT * k) : make_uint4(0, 0, 0, 0);
                    if (r0 + kOCT / 8 * k >= rows_left) x[k] = make_uint4(0, 0, 0, 0);  // past the launch: adds nothing
                }
                // The raw slot goes back to the producer with the plane stage below,
                // once the plane stores (which consume the loaded words) are done.
                const int rcur = rs;
                if (++rs == kORaws) {
                    rs = 0;
                    rph ^= 1u;
                }
                ok = mbar_wait_backoff(empty(ps), pph ^ 1u, err, kDevTimeoutProducer, XENG_CONV_SLEEP_NS);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                if (active) {
                    uint8_t *dim = sgen + (plane(ps) - sbase) + poff;  // Im plane of the tile
                    uint8_t *dre = dim + kOBox;                        // Re plane of the tile
                    #pragma unroll
                    for (int k = 0; k < kOChunks; k++) {
                        uint4 re, im;
                        re.x = (x[k].x >> 4) & 0x0F0F0F0Fu;
                        re.y = (x[k].y >> 4) & 0x0F0F0F0Fu;
                        re.z = (x[k].z >> 4) & 0x0F0F0F0Fu;
                        re.w = (x[k].w >> 4) & 0x0F0F0F0Fu;
                        im.x = x[k].x & 0x0F0F0F0Fu;
                        im.y = x[k].y & 0x0F0F0F0Fu;
                        im.z = x[k].z & 0x0F0F0F0Fu;
                        im.w = x[k].w & 0x0F0F0F0Fu;
                        *reinterpret_cast<uint4 *>(dre + 16 * kOCT * k) = re;
                        *reinterpret_cast<uint4 *>(dim + 16 * kOCT * k) = im;
                        pb[0] += re.x; pb[1] += re.y; pb[2] += re.z; pb[3] += re.w;
                        qb[0] += im.x; qb[1] += im.y; qb[2] += im.z; qb[3] += im.w;
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // planes visible to the MMAs
                }
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(full(ps));
                    mbar_arrive(rawe(rcur));
                }
                if (++ps == kOPlanes) {
                    ps = 0;
                    pph ^= 1u;
                }
                if ((kc + 1) % kOWiden == 0) widen();
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
                const int wd = m >> 2, b = m & 3;
                P32[m] = (P16[2 * wd + (b & 1)] >> (16 * (b >> 1))) & 0xFFFFu;
                Q32[m] = (Q16[2 * wd + (b & 1)] >> (16 * (b >> 1))) & 0xFFFFu;
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
            if (active && (r0 & 3) == 0) {
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
        const int q = warp & 3;                          // TMEM lane quadrant this warp may access
        constexpr int kPerQuad = kOEpiWarps / 4;         // warps of a quadrant: alternate 8-column chunks
        const int half = (warp - kOEpiWarp0) >> 2;       // this warp's first chunk
        const int et = (warp - kOEpiWarp0) * 32 + lane;
        const int row = q * 32 + lane;                   // TMEM lane: row within the tile
        const int N = a.N;                               // <= 4096: triangle offsets within a channel fit in int
        const int n128 = 128 * (int)a.nt;                // 64 n from each of the two products
        const int64_t nb2 = (int64_t)N * (N + 1) / 2;
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16);
        int local = 0;
        for (int it = it_begin; it < a.n_items; it += it_step, ++local) {
            const OnepassItem w = onepass_item(a, it);
            const int par = local & 1, ab = local & 1;  // sums buffer and accumulator
            bool ok = mbar_wait_backoff(accf(ab), (uint32_t)((local >> 1) & 1), err, kDevTimeoutEpilogue, 128);
            ok = ok && mbar_wait_backoff(sums_full(par), (uint32_t)((local >> 1) & 1), err, kDevTimeoutEpilogue, 128);
            // the barrier ORs the eight warps' failures, so they leave together
            if (bar_any(2, kOEpiWarps * 32, !ok)) break;
            fence_after();
            const bool diag = w.I == w.J;
            const int j_warp = w.J * 128 + q * 32;  // the warp's first input j (TMEM lanes: block J)
            const int j = j_warp + lane;
            const int2 *scol = sums + par * 256 + (diag ? 0 : 128);  // inputs i of the columns (block I)
            if (j_warp < N) {
                const bool lane_ok = j < N;
                const int2 pq = sums[par * 256 + row];
                const int sj = pq.x + pq.y, dj = pq.x - pq.y;
                int2 *out = reinterpret_cast<int2 *>(a.acc) + (int64_t)w.fl * nb2;
                const uint32_t tb = taddr + 256u * ab;
                const int ibase = w.I * 128;
                // Corrects the chunk of columns c..c+7 held in (vre, vim) in place and stores
                // or adds it: pair (i, j) sits at i*N - i*(i-1)/2 + (j - i) in the channel's
                // triangle and row i + 1 starts N - i - 1 pairs after row i, so per column
                // the warp's 32 consecutive inputs j are one 256-byte run.
                auto put_chunk = [&](const int c, uint32_t (&vre)[8], uint32_t (&vim)[8]) {
                    const int i0 = ibase + c;
                    #pragma unroll
                    for (int e = 0; e < 8; e++) {  // corrected values in place of the accumulator words
                        const int2 pi = scol[c + e];  // the same for every lane: a broadcast
                        // accumulators hold integer sums / 2^18 (x 2^18 is exact); with A = x_j
                        // the Im half holds minus Im of x_i conj(x_j)
                        vre[e] = (uint32_t)(__float2int_rn(262144.0f * __uint_as_float(vre[e])) -
                                            8 * (sj + pi.x + pi.y) + n128);
                        vim[e] = (uint32_t)(8 * ((pi.x - pi.y) - dj) -
                                            __float2int_rn(262144.0f * __uint_as_float(vim[e])));
                    }
                    const int off0 = i0 * N - i0 * (i0 - 1) / 2 - i0 + j;
                    const int last = min(j - i0, N - 1 - i0);  // elements e <= last are pairs of the triangle
                    if (kAdd) {
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
                auto chunk_ok = [&](const int c) { return c < 128 && ibase + c < N && ibase + c <= j_warp + 31; };
                constexpr int kStep = 8 * kPerQuad;
                if (kAdd) {  // adding to the triangle: one chunk at a time
                    for (int c = 8 * half; chunk_ok(c); c += kStep) {
                        uint32_t vre[8], vim[8];
                        tmem_ld8(tb + c, vre);
                        tmem_ld8(tb + 128u + c, vim);
                        tmem_ld_wait();
                        put_chunk(c, vre, vim);
                    }
                } else {
                    // two register sets: the next chunk's TMEM loads run under this chunk's stores
                    uint32_t ra[8], ia[8], rb[8], ib[8];
                    int c = 8 * half;
                    if (chunk_ok(c)) {
                        tmem_ld8(tb + c, ra);
                        tmem_ld8(tb + 128u + c, ia);
                    }
                    tmem_ld_wait();
                    while (chunk_ok(c)) {
                        const int c1 = c + kStep;
                        const bool ok1 = chunk_ok(c1);
                        if (ok1) {
                            tmem_ld8(tb + c1, rb);
                            tmem_ld8(tb + 128u + c1, ib);
                        }
                        put_chunk(c, ra, ia);
                        tmem_ld_wait();
                        if (!ok1) break;
                        const int c2 = c1 + kStep;
                        const bool ok2 = chunk_ok(c2);
                        if (ok2) {
                            tmem_ld8(tb + c2, ra);
                            tmem_ld8(tb + 128u + c2, ia);
                        }
                        put_chunk(c1, rb, ib);
                        tmem_ld_wait();
                        c = c2;
                    }
                }
            }
            // the accumulator is read: hand it back; every epilogue thread is done
            // with this parity's sums: clear them for the item after next
            fence_before();
            named_bar_sync(2, kOEpiWarps * 32);
            for (int k = et; k < 256; k += kOEpiWarps * 32) sums[par * 256 + k] = make_int2(0, 0);
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(acce(ab));
                mbar_arrive(sums_empty(par));
            }
        }
    }

    __syncwarp();
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kOTmemCols));
    }
}

}  // namespace

bool onepass_ok(const uint8_t *block, int32_t N)
{
    return N >= 16 && N <= 4096 && N % 16 == 0 && (reinterpret_cast<uintptr_t>(block) & 15) == 0;
}

cudaError_t encode_onepass_map(CUtensorMap *map, const uint8_t *block, int64_t T_block, int32_t F, int32_t N)
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    // raw block: dims (input, channel, sample), boxes of 128 inputs x 1 channel x kOKc
    // samples with a 128-byte swizzle (the MN-major operand layout); inputs past N and
    // samples past the block read as zero bytes, nibbles 0 that add nothing (the
    // converters zero the samples past the launch; rows and columns past N are never
    // written)
    cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)F, (cuuint64_t)T_block};
    cuuint64_t strides[2] = {(cuuint64_t)N, (cuuint64_t)N * F};
    cuuint32_t box[3] = {128, 1, (cuuint32_t)kOKc}, estr[3] = {1, 1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, (void *)block, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

int onepass_stage_samples() { return kOKc; }

cudaError_t launch_correlate_onepass(const uint8_t *block, int64_t T_block, int64_t t0, int64_t nt, int32_t F,
                                     int32_t N, int32_t f0, int32_t nf, int32_t *acc, int accumulate, int *err,
                                     int num_sms, cudaStream_t s,
                                     const CUtensorMap *maps, int32_t spb)
{
    if (nf <= 0 || nt <= 0) return cudaSuccess;
    if (!onepass_ok(maps ? nullptr : block, N) || (maps && (spb < 1 || t0 != 0)) || nt > kFusedMaxSamples ||
        t0 < 0 || t0 + nt > T_block || T_block > 2147483647LL ||
        f0 < 0 || f0 + nf > F || num_sms < 1 || (reinterpret_cast<uintptr_t>(acc) & 7) != 0)
        return cudaErrorInvalidValue;
    const int32_t nb = (N + 127) / 128;
    const int64_t n_items = (int64_t)nf * (nb * (nb + 1) / 2);
    if (n_items > 2147483647LL) return cudaErrorInvalidValue;
    CUtensorMap map;
    if (maps) {
        memset(&map, 0, sizeof map);  // not read: the stages take the blocks' maps
    } else {
        cudaError_t e0 = encode_onepass_map(&map, block, T_block, F, N);
        if (e0 != cudaSuccess) return e0;
    }
    auto kernel = accumulate ? correlate_onepass_kernel<true> : correlate_onepass_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOSmem);
    if (e != cudaSuccess) return e;
    OnepassArgs a;
    a.t0 = t0;
    a.nt = nt;
    a.F = F;
    a.N = N;
    a.f0 = f0;
    a.nf = nf;
    a.nb = nb;
    a.pairs_per_ch = nb * (nb + 1) / 2;
    a.n_items = (int32_t)n_items;
    a.acc = acc;
    a.accumulate = accumulate;
    a.err = err;
    a.maps = maps;
    a.spb = spb;
    const int grid = n_items < num_sms ? (int)n_items : num_sms;
    kernel<<<grid, kOThreads, kOSmem, s>>>(map, a);
    return cudaGetLastError();
}

}  // namespace xeng
