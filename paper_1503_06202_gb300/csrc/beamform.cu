// beamform.cu -- discrete beamforming on the tensor cores (paper Sec. IV-C-3:
// the data of all inputs are phase-shifted and summed, so that signals from
// a chosen sky direction add in phase; the beam is written out at the full
// sample cadence).
//
// For every sample t, channel f and beam b
//     y_b(t, f) = sum_i w_{f,b,i} x_i(t, f),
// x_i decoded from the 4+4-bit offset bytes (Sec. II-A), w = w_re + i w_im
// with int8 parts.  As real GEMMs with M = 128 samples and K = inputs:
//     Re y = X_re W_re^T - X_im W_im^T,   Im y = X_re W_im^T + X_im W_re^T.
// The samples enter undecoded: each nibble u (0..15) is the FP6 E2M3 code of
// u / 8 (see raw4_to_e2m3_pairs), and with x = u - 8
//     Re y = sum_i (w_re u_re - w_im u_im) - 8 sum_i (w_re - w_im),
//     Im y = sum_i (w_re u_im + w_im u_re) - 8 sum_i (w_re + w_im),
// whose second terms, one pair per (channel, beam), are computed once with
// the weights.  E2M3 holds the integers -15..15 / 8 but not all of int8, so a
// weight part v is split into v = 16 hi + lo, hi = v >> 4 in [-8, 8], lo =
// v & 15 in [0, 15], each the E2M3 code of part / 8.  The A operand
// interleaves the parts of each input along K (K position 2i holds Im u_i,
// 2i + 1 holds Re u_i: the order of the bytes' nibbles), so one MMA per 32 K
// positions covers both; the B operand's rows are the hi parts of the Re-y
// weights (-w_im, w_re interleaved), of the Im-y weights (w_re, w_im), then
// the lo parts of both (4 Bp rows, Bp = beams rounded up), and one 128 x 4Bp
// f32 accumulator collects the hi and lo parts of Re y and Im y side by side;
// the epilogue forms y = 64 (16 hi + lo) - correction in int32 (reading the
// scaled integers out of the float bits, see the epilogue).  Products are u v / 64 with u v an integer of magnitude <= 15 * 15
// and partial sums stay below 450 N / 64 (N <= 4096: 450 N < 2^24), so the
// f32 accumulation is exact.
//
// One persistent CTA per SM; work items = (channel, 128-sample tile):
//   warp 0        TMA producer of the 128-input slices of both weight
//                 operands (L2-resident) into a deep shared-memory ring
//   warp 1        TMEM allocation and the single-thread MMA issuer; the MMA
//                 reads its A operand (the decoded samples) from tensor memory
//                 and only B (the weights) from shared memory
//   warps 2..13   converters in three groups of four warps (one per TMEM lane
//                 quadrant); group g takes the steps g, g + 3, ...: each thread
//                 reads one sample row (128 inputs) of the step's raw tile from
//                 shared memory, splits it into E2M3 nibble codes and writes them,
//                 real and imaginary parts interleaved along K, into the
//                 group's TMEM slot with tcgen05.st
//   warps 14..17  epilogue: TMEM -> int32 beams [T][F][B][2] in HBM
//   warp 18       TMA producer of the raw tiles (128 samples x 128 inputs of one
//                 channel, 128-byte swizzle) into a six-slot ring
// Shared memory then carries only the weight slices; decoded planes written to
// and read back from shared memory made the MMAs shared-memory bound at small
// beam counts.  Two TMEM accumulators (one above 32 beams) let the epilogue of
// one item overlap the next item's MMAs.  Every wait is bounded; on time-out the roles leave their loops, the
// producer lets its issued copies land, the MMA thread drains and TMEM is
// freed before exit.
#include <cstring>
#include <new>

#include "../../include/xeng.h"
#include "nibble.cuh"
#include "tc_ptx.cuh"
#include "xeng_internal.h"

namespace xeng {
namespace {

// Converter groups: four warps each, one per TMEM lane quadrant; group g
// converts the steps n = g, g + kGroups, ... into its own TMEM slot g (a slot
// used by one group only, in order, so its barriers never run two phases apart).
constexpr int kGroups = 3;
constexpr int kConvWarps = 4 * kGroups;              // warps 2 .. 13
constexpr int kEpiWarp0 = 2 + kConvWarps;            // 4 epilogue warps (one per TMEM lane quadrant)
constexpr int kRawProdWarp = kEpiWarp0 + 4;          // TMA producer of the raw tiles
constexpr int kBfThreads = 32 * (kRawProdWarp + 1);
constexpr int kRawBytes = 128 * 128;                 // 128 samples x 128 inputs of one channel
// Raw-tile ring slots asked for (a build parameter); each configuration takes
// the largest multiple of the groups up to this that leaves two weight stages.
#ifndef XENG_BF_RAW_SLOTS
#define XENG_BF_RAW_SLOTS 6
#endif
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kXCols = 64;                      // one K chunk of 128 inputs: 256 codes, 4 to a column
constexpr float kMagic = 196608.0f;                  // 1.5 * 2^17: its binade has the spacing 2^-6
constexpr uint32_t kMagicBits = 0x48400000u;         // bit pattern of kMagic

template <int kBp>
struct BfCfg {
    static constexpr int kN = 4 * kBp;                           // MMA N: hi/lo x Re/Im x beams
    static constexpr int kWBytes = kN * 128;                     // one 128-byte-wide box of the weight operand
    static constexpr int kWStageBytes = 2 * kWBytes;             // the weight operand of one K chunk (256 K positions)
    static constexpr int kAcc = (8 * kBp <= 256) ? 2 : 1;        // accumulators (2: epilogue overlaps MMAs)
    static constexpr uint32_t kXCol0 = kAcc * kN;                // first TMEM column of the X slots
    // X slots per group: two where TMEM has room (the group converts its next
    // step while the MMAs of the previous one run), else one
    static constexpr int kSlots = (kTmemCols - kXCol0) / (kGroups * kXCols) >= 2 ? 2 : 1;
    static_assert(kXCol0 + kGroups * kSlots * kXCols <= kTmemCols, "TMEM: accumulators + X slots");
    // raw ring: a multiple of the groups, so each slot has one user
    static constexpr int kRFit = (232448 - 1024 - 512 - 2 * kBp * 8 - 2 * kWStageBytes) / kRawBytes / kGroups * kGroups;
    static constexpr int kRWant = XENG_BF_RAW_SLOTS / kGroups * kGroups;
    static constexpr int kR = kRWant < kRFit ? kRWant : kRFit;
    static_assert(kR >= kGroups, "raw ring needs a slot per converter group");
    static constexpr int kCorrBytes = 2 * kBp * 8;                // offset terms of two items, staged for the epilogue
    static constexpr int kSWFit = (232448 - 1024 - 512 - kCorrBytes - kR * kRawBytes) / kWStageBytes;
    static constexpr int kSW = kSWFit > 8 ? 8 : kSWFit;          // weight ring stages (L2 latency off the path)
    static_assert(kSW >= 2, "weight ring needs two stages");
    static constexpr int kXS = kGroups * kSlots;                 // X slots in all
    static constexpr int kBars = 2 * kR + 2 * kXS + 2 * kSW + 2 * kAcc + 1;
    static constexpr size_t kSmem =
        1024 + (size_t)kR * kRawBytes + (size_t)kSW * kWStageBytes + kBars * 8 + 16 + 8 + kCorrBytes;
    // kind::f8f6f4, D f32, A and B E2M3 (type 3) K-major, N and M = 128
    static constexpr uint32_t kIdesc = (1u << 4) | (3u << 7) | (3u << 10) | ((uint32_t)(kN >> 3) << 17) |
                                       ((uint32_t)(128 >> 4) << 24);
    static_assert(kSmem <= 232448, "shared memory over the per-CTA limit");
};

// K-major operand with 128-byte rows, 128-byte swizzle, 8-row groups 1 KB apart.
__device__ __forceinline__ uint64_t bf_desc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// MMA with A (M = 128 rows x K = 32 codes) read from tensor memory.
__device__ __forceinline__ void mma_f8_ta(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}"
        ::"r"(d), "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

__device__ __forceinline__ void bf_item(const BfArgs &a, int64_t it, int &f, int &tt)
{
    if (a.f_fastest) {
        f = (int)(it % a.F);
        tt = (int)(it / a.F);
    } else {
        tt = (int)(it % a.n_tt);
        f = (int)(it / a.n_tt);
    }
}

template <int kBp>
__global__ void __launch_bounds__(kBfThreads, 1)
beamform_kernel(const __grid_constant__ CUtensorMap raw_map, const __grid_constant__ CUtensorMap w_map, const BfArgs a)
{
    using C = BfCfg<kBp>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t rbase = (raw + 1023u) & ~1023u;                  // raw ring
    const uint8_t *rgen = smem_raw + (rbase - raw);                 // generic view of it
    const uint32_t wbase = rbase + C::kR * kRawBytes;                  // weight ring
    const uint32_t bars = wbase + C::kSW * C::kWStageBytes;
    auto xf = [&](int x) { return bars + 8u * x; };                           // X slot x written
    auto xe = [&](int x) { return bars + 8u * (C::kXS + x); };                // X slot x consumed
    auto wf = [&](int s) { return bars + 8u * (2 * C::kXS + s); };            // weight slices landed
    auto we = [&](int s) { return bars + 8u * (2 * C::kXS + C::kSW + s); };   // weight slices consumed
    auto accf = [&](int b) { return bars + 8u * (2 * C::kXS + 2 * C::kSW + b); };
    auto acce = [&](int b) { return bars + 8u * (2 * C::kXS + 2 * C::kSW + C::kAcc + b); };
    const uint32_t drain_bar = bars + 8u * (2 * C::kXS + 2 * C::kSW + 2 * C::kAcc);
    auto rawf = [&](int r) { return bars + 8u * (2 * C::kXS + 2 * C::kSW + 2 * C::kAcc + 1 + r); };       // tile landed
    auto rawe = [&](int r) { return bars + 8u * (2 * C::kXS + 2 * C::kSW + 2 * C::kAcc + 1 + C::kR + r); };  // tile read
    // step n of this CTA belongs to group n % kGroups, which uses its slots in
    // turn: slot (n / kGroups) % kSlots of the group, phase (n / kGroups / kSlots) & 1
    auto xslot = [&](int64_t n) { return (int)(n % kGroups) * C::kSlots + (int)((n / kGroups) % C::kSlots); };
    auto xphase = [&](int64_t n) { return (uint32_t)((n / kGroups / C::kSlots) & 1); };
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem_raw + (bars + 8u * C::kBars - raw));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *err = a.err;
    const int64_t n_seq = ((a.n_items - blockIdx.x + gridDim.x - 1) / gridDim.x) * a.n_kc;

    if (threadIdx.x == 0) {
        for (int x = 0; x < C::kXS; x++) {
            mbar_init(xf(x), 128);
            mbar_init(xe(x), 1);
        }
        for (int s = 0; s < C::kSW; s++) {
            mbar_init(wf(s), 1);
            mbar_init(we(s), 1);
        }
        for (int b = 0; b < C::kAcc; b++) {
            mbar_init(accf(b), 1);
            mbar_init(acce(b), 128);
        }
        mbar_init(drain_bar, 1);
        for (int r = 0; r < C::kR; r++) {
            mbar_init(rawf(r), 1);
            mbar_init(rawe(r), 128);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&w_map) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&raw_map) : "memory");
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
            // ---------------- TMA producer: weight slices ----------------
            int s = 0, issued = 0;
            uint32_t ps = 0;
            bool ok = true;
            for (int64_t it = blockIdx.x; ok && it < a.n_items; it += gridDim.x) {
                int f, tt;
                bf_item(a, it, f, tt);
                for (int k = 0; k < a.n_kc; k++) {
                    if (!mbar_wait(we(s), ps ^ 1u, err, kDevTimeoutProducer)) {
                        ok = false;
                        break;
                    }
                    // K positions 256k .. 256k + 255 (inputs 128k .. 128k + 127) as two
                    // 128-byte-swizzled boxes
                    const uint32_t w0 = wbase + s * C::kWStageBytes;
                    mbar_expect_tx(wf(s), 2 * C::kWBytes);
                    tma_load_2d(w0, &w_map, k * 256, f * C::kN, wf(s));
                    tma_load_2d(w0 + C::kWBytes, &w_map, k * 256 + 128, f * C::kN, wf(s));
                    ++issued;
                    if (++s == C::kSW) {
                        s = 0;
                        ps ^= 1u;
                    }
                }
            }
            if (!ok) {
                // Let the copies already issued land before the CTA can exit.
                for (int k = 1; k <= C::kSW && k <= issued; k++) {
                    int q = s - k, p = (int)ps;
                    if (q < 0) { q += C::kSW; p ^= 1; }
                    (void)mbar_wait(wf(q), (uint32_t)p, err, kDevTimeoutProducer);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            // Per step: two waits, eight MMAs, two commits; the bookkeeping is
            // kept to a few integer operations since each step carries little
            // tensor work (N = 4 Bp).
            int sw = 0, local = 0, c = 0;  // c = step index modulo the X slots
            uint32_t pw = 0, pxs = 0;
            bool ok = true;
            for (int64_t it = blockIdx.x; ok && it < a.n_items; it += gridDim.x, ++local) {
                const int ab = C::kAcc == 2 ? (local & 1) : 0;
                // the accumulator's earlier uses: local / kAcc (a counter array indexed by ab would live in local memory)
                const uint32_t used = (uint32_t)(C::kAcc == 2 ? (local >> 1) : local);
                if (!mbar_wait_backoff(acce(ab), (used & 1u) ^ 1u, err, kDevTimeoutMma, 0)) break;
                fence_after();
                const uint32_t d = tmem + (uint32_t)(ab * C::kN);
                for (int k = 0; k < a.n_kc; k++) {
                    const int x = (c % kGroups) * C::kSlots + c / kGroups;
                    if (!mbar_wait_backoff(wf(sw), pw, err, kDevTimeoutMma, 0) ||
                        !mbar_wait_backoff(xf(x), pxs, err, kDevTimeoutMma, 0)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t xs = tmem + C::kXCol0 + (uint32_t)x * kXCols;
                    const uint32_t w0 = wbase + sw * C::kWStageBytes;
                    const uint64_t b0 = bf_desc(w0), b1 = bf_desc(w0 + C::kWBytes);
                    #pragma unroll
                    for (int kk = 0; kk < 8; kk++) {  // +32 bytes along K = +2 in the descriptor's address field
                        const uint64_t bk = (kk < 4 ? b0 : b1) + 2 * (kk & 3);
                        mma_f8_ta(d, xs + kk * 8, bk, C::kIdesc, (k != 0 || kk != 0) ? 1u : 0u);
                    }
                    mma_commit(xe(x));
                    mma_commit(we(sw));
                    if (++sw == C::kSW) {
                        sw = 0;
                        pw ^= 1u;
                    }
                    if (++c == C::kXS) {
                        c = 0;
                        pxs ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit(accf(ab));
            }
            // Drain: every MMA issued above has finished once this completes.
            mma_commit(drain_bar);
            (void)mbar_wait(drain_bar, 0u, err, kDevTimeoutMma);
        }
    } else if (warp < kEpiWarp0) {
        // ---------------- converters: raw tile (smem) -> E2M3 nibble codes in TMEM ----------------
        // Thread = one sample row of a step (its TMEM lane): the row's 128
        // bytes from the 128-byte-swizzled raw tile (conflict-free: lanes t and
        // t + 8 share a chunk position, the minimum for 16-byte reads).
        const int g = (warp - 2) >> 2;
        const int q = warp & 3;  // TMEM lane quadrant this warp may access
        const int row = q * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16) + C::kXCol0;
        for (int64_t n = g; n < n_seq; n += kGroups) {
            const int r = (int)(n % C::kR);
            const uint32_t pr = (uint32_t)((n / C::kR) & 1);
            const int x = xslot(n);
            const bool ok = mbar_wait_backoff(rawf(r), pr, err, kDevTimeoutProducer, XENG_CONV_SLEEP_NS) &&
                            mbar_wait_backoff(xe(x), xphase(n) ^ 1u, err, kDevTimeoutProducer, XENG_CONV_SLEEP_NS);
            if (!__all_sync(0xffffffffu, ok)) break;  // keep the warp converged for tcgen05.st
            fence_after();
            const uint8_t *rt = rgen + r * kRawBytes + row * 128;
            uint4 v[8];
            #pragma unroll
            for (int j = 0; j < 8; j++) v[j] = *reinterpret_cast<const uint4 *>(rt + ((j ^ (row & 7)) << 4));
            mbar_arrive(rawe(r));
            const uint32_t xs = lane_base + (uint32_t)x * kXCols;
            #pragma unroll
            for (int h = 0; h < 8; h++) {  // 16 inputs = 8 columns of (Im, Re) codes per store
                const uint4 w = v[h];
                const uint32_t wd[4] = {w.x, w.y, w.z, w.w};
                uint32_t col[8];
                #pragma unroll
                for (int j = 0; j < 4; j++)  // inputs 4j .. 4j + 3 of the 16: (Im, Re) of 4j, 4j + 1 | 4j + 2, 4j + 3
                    raw4_to_e2m3_pairs(wd[j], col[2 * j], col[2 * j + 1]);
                tmem_st8(xs + h * 8, col);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            fence_before();
            mbar_arrive(xf(x));
        }
    } else if (warp < kRawProdWarp) {
        // ---------------- epilogue (warps 14..17) ----------------
        // The offset terms of an item's channel are loaded by the first
        // epilogue warp while the MMAs run and staged in shared memory (two
        // items' worth, alternating), where the four warps read them as
        // broadcasts; a barrier over the four warps publishes them and also
        // ORs the warps' wait results, so that all four leave together.
        const int q = warp & 3;  // TMEM lane quadrant this warp may access
        const int row = q * 32 + lane;
        const bool stager = warp == kEpiWarp0;
        // [2][kBp], 16-byte aligned for the paired loads (the barrier area ends 8 bytes off a 16-byte boundary
        // when the barrier count is odd)
        int2 *corr_s = reinterpret_cast<int2 *>(smem_raw + (((bars + 8u * C::kBars + 16 + 15) & ~15u) - raw));
        constexpr int G = kBp < 16 ? kBp : 16;
        constexpr int kPer = (kBp + 31) / 32;  // offset terms per lane of the staging warp
        int local = 0;
        for (int64_t it = blockIdx.x; it < a.n_items; it += gridDim.x, ++local) {
            int f, tt;
            bf_item(a, it, f, tt);
            const int ab = C::kAcc == 2 ? (local & 1) : 0;
            int2 cv[kPer];
            if (stager) {
                const int2 *corr = reinterpret_cast<const int2 *>(a.corr) + (int64_t)f * kBp;
                #pragma unroll
                for (int k = 0; k < kPer; k++)
                    if (lane + 32 * k < kBp) {
                        const int2 c = __ldg(corr + lane + 32 * k);
                        // with the conversion offsets of the hi (x 16) and lo parts folded in
                        cv[k] = make_int2((int)((uint32_t)c.x + 17u * kMagicBits), (int)((uint32_t)c.y + 17u * kMagicBits));
                    }
            }
            const uint32_t used = (uint32_t)(C::kAcc == 2 ? (local >> 1) : local);  // the accumulator's earlier uses
            const bool ok = mbar_wait_backoff(accf(ab), used & 1u, err, kDevTimeoutEpilogue, 256);
            int2 *cs = corr_s + (local & 1) * kBp;
            if (stager) {
                // the slot was last read two items ago, before the previous item's barrier
                #pragma unroll
                for (int k = 0; k < kPer; k++)
                    if (lane + 32 * k < kBp) cs[lane + 32 * k] = cv[k];
            }
            uint32_t any_fail;
            asm volatile(
                "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
                "bar.red.or.pred p, 1, 128, q;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(any_fail)
                : "r"(ok ? 0u : 1u)
                : "memory");
            if (any_fail) break;  // all four warps, converged for tcgen05.ld
            fence_after();
            const int64_t t = (int64_t)tt * 128 + row;
            int2 *o = reinterpret_cast<int2 *>(a.out) + (t * a.F + f) * a.B;
            int4 *o4 = reinterpret_cast<int4 *>(o);  // two beams per store when B is even
            const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * C::kN);
            #pragma unroll
            for (int b0 = 0; b0 < kBp; b0 += G) {
                uint32_t hre[G], him[G], lre[G], lim[G];
                #pragma unroll
                for (int c = 0; c < G; c += 4) {
                    tmem_ld4(ta + b0 + c, *reinterpret_cast<uint32_t(*)[4]>(hre + c));
                    tmem_ld4(ta + kBp + b0 + c, *reinterpret_cast<uint32_t(*)[4]>(him + c));
                    tmem_ld4(ta + 2 * kBp + b0 + c, *reinterpret_cast<uint32_t(*)[4]>(lre + c));
                    tmem_ld4(ta + 3 * kBp + b0 + c, *reinterpret_cast<uint32_t(*)[4]>(lim + c));
                }
                tmem_ld_wait();
                if (t < a.T) {
                    // An accumulator holds S / 64 for an integer |S| < 2^22; adding 1.5 * 2^17
                    // (ulp 2^-6) is exact and leaves S + kMagicBits in the sum's bit pattern,
                    // so y = 16 S_hi + S_lo - offset needs no float-to-int conversion.
                    int2 y[G];
                    #pragma unroll
                    for (int e = 0; e < G; e++) {
                        int2 c;
                        if (G >= 2) {  // two beams' offset terms per shared-memory load
                            const int4 c2 = *reinterpret_cast<const int4 *>(cs + b0 + (e & ~1));
                            c = (e & 1) ? make_int2(c2.z, c2.w) : make_int2(c2.x, c2.y);
                        } else {
                            c = cs[b0 + e];
                        }
                        const uint32_t bhr = __float_as_uint(__uint_as_float(hre[e]) + kMagic);
                        const uint32_t blr = __float_as_uint(__uint_as_float(lre[e]) + kMagic);
                        const uint32_t bhi = __float_as_uint(__uint_as_float(him[e]) + kMagic);
                        const uint32_t bli = __float_as_uint(__uint_as_float(lim[e]) + kMagic);
                        y[e] = make_int2((int)(16u * bhr + blr - (uint32_t)c.x), (int)(16u * bhi + bli - (uint32_t)c.y));
                    }
                    if (a.vec16) {
                        #pragma unroll
                        for (int e = 0; e < G; e += 2)
                            if (b0 + e < a.B) o4[(b0 + e) >> 1] = make_int4(y[e].x, y[e].y, y[e + 1].x, y[e + 1].y);
                    } else {
                        #pragma unroll
                        for (int e = 0; e < G; e++)
                            if (b0 + e < a.B) o[b0 + e] = y[e];
                    }
                }
            }
            fence_before();
            mbar_arrive(acce(ab));
        }
    } else if (lane == 0) {
        // ---------------- TMA producer: raw tiles (warp 18) ----------------
        int issued = 0;
        bool ok = true;
        for (int64_t n = 0; n < n_seq; n++) {
            const int r = (int)(n % C::kR);
            if (!mbar_wait(rawe(r), (uint32_t)((n / C::kR) & 1) ^ 1u, err, kDevTimeoutProducer)) {
                ok = false;
                break;
            }
            const int64_t it = blockIdx.x + (n / a.n_kc) * (int64_t)gridDim.x;
            int f, tt;
            bf_item(a, it, f, tt);
            mbar_expect_tx(rawf(r), kRawBytes);
            tma_load_3d(rbase + r * kRawBytes, &raw_map, (int)(n % a.n_kc) * 128, f, tt * 128, rawf(r));
            ++issued;
        }
        if (!ok) {
            // Let the copies already issued land before the CTA can exit.
            for (int64_t n = issued - 1; n >= 0 && n >= issued - C::kR; n--)
                (void)mbar_wait(rawf((int)(n % C::kR)), (uint32_t)((n / C::kR) & 1), err, kDevTimeoutProducer);
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

// Weight operand from int8 weights [F][B][N] (re, im): [F][4 Bp][2 n_pad]
// bytes; row g * Bp + b holds the hi (g = 0, 1) or lo (g = 2, 3) part of the
// Re-y (g even) or Im-y (g odd) weights of beam b, K position 2i the factor of
// Im x_i and 2i + 1 that of Re x_i.  Rows b >= B and inputs i >= N are zero.
// Each part v (|v| <= 15) is the E2M3 code of v / 8 (sign bit 5, |v| in bits
// 0..3).  In shared memory the tensor core reads an FP6 operand as 16 codes
// packed in the first 12 bytes of each 16-byte chunk (code j in bits 6j ..
// 6j + 5, little-endian) followed by 4 unused bytes -- measured on GB300 --
// so each thread packs one chunk of 16 K positions; the chunk grid, and so
// the tensor-map boxes and the swizzle, are those of one byte per element.
__global__ void beam_weights_kernel(const int8_t *__restrict__ w_re, const int8_t *__restrict__ w_im, int32_t F,
                                    int32_t B, int32_t N, int32_t bp, int32_t n_pad, uint4 *__restrict__ wdev)
{
    const int chunks_per_row = (2 * n_pad) / 16;
    const int64_t total = (int64_t)F * 4 * bp * chunks_per_row;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(k % chunks_per_row);
        const int64_t rowk = k / chunks_per_row;
        const int rr = (int)(rowk % (4 * bp));
        const int64_t f = rowk / (4 * bp);
        const int g = rr / bp, b = rr % bp;
        uint64_t lo = 0, hi = 0;  // bits 0..63 and 64..95 of the packed chunk
        for (int j = 0; j < 16; j++) {
            const int kp = ch * 16 + j;
            const int i = kp >> 1;
            const bool of_re = (kp & 1) != 0;  // multiplies Re x_i (else Im x_i)
            int v = 0;
            if (b < B && i < N) {
                const int64_t src = (f * B + b) * N + i;
                const int wr = w_re[src], wi = w_im[src];
                // Re y += Re x w_re - Im x w_im;  Im y += Re x w_im + Im x w_re
                const int base = (g & 1) ? (of_re ? wi : wr) : (of_re ? wr : -wi);
                v = g < 2 ? (base >> 4) : (base & 15);
            }
            const uint64_t code = (uint64_t)(v < 0 ? (0x20 | -v) : v);
            const int bit = 6 * j;
            if (bit < 64) lo |= code << bit;
            if (bit >= 64)
                hi |= code << (bit - 64);
            else if (bit + 6 > 64)
                hi |= code >> (64 - bit);  // the code straddling bit 64
        }
        wdev[k] = make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, 0u);
    }
}

// Offset terms per (channel, beam): corr[f][b] = (8 sum_i (w_re - w_im),
// 8 sum_i (w_re + w_im)), zero for padding beams b >= B.  One block per
// (channel, padded beam).
__global__ void beam_corr_kernel(const int8_t *__restrict__ w_re, const int8_t *__restrict__ w_im, int32_t B,
                                 int32_t N, int32_t bp, int2 *__restrict__ corr)
{
    const int64_t fb = blockIdx.x;
    const int b = (int)(fb % bp);
    const int64_t f = fb / bp;
    int sre = 0, sim = 0;
    if (b < B) {
        const int64_t src = (f * B + b) * N;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const int wr = w_re[src + i], wi = w_im[src + i];
            sre += wr - wi;
            sim += wr + wi;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sre += __shfl_xor_sync(0xffffffffu, sre, o);
        sim += __shfl_xor_sync(0xffffffffu, sim, o);
    }
    __shared__ int red[2][32];
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sre;
        red[1][threadIdx.x >> 5] = sim;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int r0 = 0, r1 = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
            r0 += red[0][k];
            r1 += red[1][k];
        }
        corr[fb] = make_int2(8 * r0, 8 * r1);
    }
}

template <int kBp>
cudaError_t launch_bf(const CUtensorMap &rm, const CUtensorMap &wm, const BfArgs &a, int grid, cudaStream_t s)
{
    using C = BfCfg<kBp>;
    cudaError_t e = cudaFuncSetAttribute(beamform_kernel<kBp>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::kSmem);
    if (e != cudaSuccess) return e;
    beamform_kernel<kBp><<<grid, kBfThreads, C::kSmem, s>>>(rm, wm, a);
    return cudaGetLastError();
}

}  // namespace

int beam_padded(int32_t n_beams)
{
    return n_beams <= 4 ? 4 : n_beams <= 8 ? 8 : n_beams <= 16 ? 16 : n_beams <= 32 ? 32 : 64;
}

cudaError_t launch_beam_weights(const int8_t *w_re, const int8_t *w_im, int32_t F, int32_t B, int32_t N,
                                uint8_t *wdev, int32_t *corr, cudaStream_t s)
{
    const int bp = beam_padded(B);
    const int n_pad = (int)round_up(N, 128);
    const int64_t total = (int64_t)F * 8 * bp * n_pad / 16;  // 16-position chunks of F x 4 Bp rows x 2 n_pad
    int64_t blocks = (total + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    beam_weights_kernel<<<(unsigned)blocks, 256, 0, s>>>(w_re, w_im, F, B, N, bp, n_pad,
                                                         reinterpret_cast<uint4 *>(wdev));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    beam_corr_kernel<<<(unsigned)((int64_t)F * bp), 128, 0, s>>>(w_re, w_im, B, N, bp, reinterpret_cast<int2 *>(corr));
    return cudaGetLastError();
}

cudaError_t launch_beamform(const uint8_t *block, const uint8_t *wdev, const int32_t *corr, BfArgs a, int num_sms,
                            cudaStream_t s)
{
    if (a.T <= 0) return cudaSuccess;
    a.corr = corr;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    const int bp = beam_padded(a.B);
    const int n_pad = (int)round_up(a.N, 128);
    // raw block: dims (input, channel, sample), boxes of 128 inputs x 1 channel
    // x 128 samples, 128-byte swizzle (conflict-free row reads by the converters)
    CUtensorMap rm, wm;
    {
        cuuint64_t dims[3] = {(cuuint64_t)a.N, (cuuint64_t)a.F, (cuuint64_t)a.T};
        cuuint64_t strides[2] = {(cuuint64_t)a.N, (cuuint64_t)a.N * a.F};
        cuuint32_t box[3] = {128, 1, 128}, estr[3] = {1, 1, 1};
        if (enc(&rm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, (void *)block, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        // weights [F][4 Bp][2 n_pad]: boxes of 128 K positions x 4 Bp rows
        cuuint64_t dims[2] = {(cuuint64_t)(2 * n_pad), (cuuint64_t)a.F * 4 * bp};
        cuuint64_t strides[1] = {(cuuint64_t)(2 * n_pad)};
        cuuint32_t box[2] = {128, (cuuint32_t)(4 * bp)}, estr[2] = {1, 1};
        if (enc(&wm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void *)wdev, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    a.n_kc = n_pad / 128;
    a.n_tt = (int32_t)((a.T + 127) / 128);
    a.n_items = (int64_t)a.F * a.n_tt;
    // channel-fastest order reads neighbouring channels' rows together; it
    // needs every channel's weights in L2, else one channel at a time
    a.f_fastest = ((int64_t)a.F * 8 * bp * n_pad <= ((int64_t)48 << 20)) ? 1 : 0;
    a.block = block;
    a.vec16 = (a.B % 2 == 0 && (reinterpret_cast<uintptr_t>(a.out) & 15) == 0) ? 1 : 0;
    const int grid = (int)(a.n_items < num_sms ? a.n_items : num_sms);
    switch (bp) {
        case 4: return launch_bf<4>(rm, wm, a, grid, s);
        case 8: return launch_bf<8>(rm, wm, a, grid, s);
        case 16: return launch_bf<16>(rm, wm, a, grid, s);
        case 32: return launch_bf<32>(rm, wm, a, grid, s);
        default: return launch_bf<64>(rm, wm, a, grid, s);
    }
}

}  // namespace xeng

// ---------------------------------------------------------------------------
// C ABI
struct xbeam_s {
    int32_t N = 0, F = 0, B = 0;
    int device = 0, num_sms = 0;
    uint8_t *wdev = nullptr;    // [F][4 Bp][2 n_pad] E2M3 weight operand
    int64_t wdev_bytes = 0;
    int32_t *corr = nullptr;    // [F][Bp][2] offset terms of the beams
    int8_t *wstage = nullptr;   // device copy of host weights
    int *d_err = nullptr;       // device status word of the kernels
    int *h_err = nullptr;       // pinned mirror, refreshed after each run
    int sticky = XENG_OK;
};

namespace {

bool bf_is_device_pointer(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int bf_status(cudaError_t e)
{
    if (e == cudaSuccess) return XENG_OK;
    if (e == cudaErrorMemoryAllocation) return XENG_ERR_NOMEM;
    return XENG_ERR_CUDA;
}

int bf_check_sticky(xbeam_s *b)
{
    if (b->sticky != XENG_OK) return b->sticky;
    if (*b->h_err != 0) b->sticky = XENG_ERR_TIMEOUT;
    return b->sticky;
}

}  // namespace

extern "C" {

int xbeam_create(int32_t n_inputs, int32_t n_freq, int32_t n_beams, xbeam_t *out)
{
    if (!out) return XENG_ERR_ARG;
    *out = nullptr;
    if (n_inputs < 16 || n_inputs > XENG_MAX_INPUTS || n_inputs % 16 != 0 || n_freq < 1 || n_beams < 1 ||
        n_beams > XBEAM_MAX_BEAMS)
        return XENG_ERR_RANGE;
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return XENG_ERR_UNSUPPORTED;
    }
    if (prop.major != 10 || prop.minor != 3) return XENG_ERR_UNSUPPORTED;
    xbeam_s *b = new (std::nothrow) xbeam_s;
    if (!b) return XENG_ERR_NOMEM;
    b->N = n_inputs;
    b->F = n_freq;
    b->B = n_beams;
    b->device = dev;
    b->num_sms = prop.multiProcessorCount;
    b->wdev_bytes = (int64_t)n_freq * 8 * xeng::beam_padded(n_beams) * xeng::round_up(n_inputs, 128);
    cudaError_t e = cudaMalloc(&b->wdev, (size_t)b->wdev_bytes);
    if (e == cudaSuccess) e = cudaMemset(b->wdev, 0, (size_t)b->wdev_bytes);  // E2M3 +0: all weights zero
    const size_t corr_bytes = (size_t)n_freq * xeng::beam_padded(n_beams) * 2 * sizeof(int32_t);
    if (e == cudaSuccess) e = cudaMalloc(&b->corr, corr_bytes);
    if (e == cudaSuccess) e = cudaMemset(b->corr, 0, corr_bytes);  // and so are their offset terms
    if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_err, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        xbeam_destroy(b);
        return bf_status(e);
    }
    *b->h_err = 0;
    *out = b;
    return XENG_OK;
}

int xbeam_set_weights(xbeam_t b, const int8_t *w_re, const int8_t *w_im, void *stream)
{
    if (!b || !w_re || !w_im) return XENG_ERR_ARG;
    int st = bf_check_sticky(b);
    if (st != XENG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = (int64_t)b->F * b->B * b->N;
    const bool dre = bf_is_device_pointer(w_re), dim = bf_is_device_pointer(w_im);
    cudaError_t e = cudaSuccess;
    if (!dre || !dim) {
        if (!b->wstage) {
            e = cudaMalloc(&b->wstage, (size_t)(2 * n));
            if (e != cudaSuccess) {
                cudaGetLastError();
                b->wstage = nullptr;
                return XENG_ERR_NOMEM;
            }
        }
        if (!dre) e = cudaMemcpyAsync(b->wstage, w_re, (size_t)n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !dim) e = cudaMemcpyAsync(b->wstage + n, w_im, (size_t)n, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return (b->sticky = bf_status(e));
    }
    e = xeng::launch_beam_weights(dre ? w_re : b->wstage, dim ? w_im : b->wstage + n, b->F, b->B, b->N, b->wdev,
                                  b->corr, s);
    // host weights may be reused by the caller at once
    if (e == cudaSuccess && (!dre || !dim)) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return (b->sticky = bf_status(e));
    return XENG_OK;
}

int xbeam_run(xbeam_t b, const uint8_t *block, int64_t n_samples, int32_t *out, void *stream)
{
    if (!b || n_samples < 0) return XENG_ERR_ARG;
    int st = bf_check_sticky(b);
    if (st != XENG_OK) return st;
    if (n_samples == 0) return XENG_OK;
    if (n_samples > ((int64_t)1 << 31) - 128) return XENG_ERR_RANGE;
    if (!block || !out || !bf_is_device_pointer(block) || !bf_is_device_pointer(out)) return XENG_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(block) & 15) != 0 || (reinterpret_cast<uintptr_t>(out) & 7) != 0)
        return XENG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    xeng::BfArgs a;
    a.T = n_samples;
    a.F = b->F;
    a.N = b->N;
    a.B = b->B;
    a.out = out;
    a.err = b->d_err;
    cudaError_t e = xeng::launch_beamform(block, b->wdev, b->corr, a, b->num_sms, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return (b->sticky = bf_status(e));
    return XENG_OK;
}

void xbeam_destroy(xbeam_t b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    cudaFree(b->wdev);
    cudaFree(b->corr);
    cudaFree(b->wstage);
    cudaFree(b->d_err);
    if (b->h_err) cudaFreeHost(b->h_err);
    cudaGetLastError();
    delete b;
}

}  // extern "C"
