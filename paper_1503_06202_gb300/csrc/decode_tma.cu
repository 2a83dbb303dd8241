// decode_tma.cu -- the decode stage (paper Sec. II-A: nibble = value + 8,
// high nibble real, low nibble imaginary) as a persistent TMA pipeline: the
// same planes as decode_kernel ([nf][2][n_pad][t_pad] E4M3 codes, K-major,
// +0.0 outside the block), for blocks whose rows TMA can address (N a multiple
// of 16, block 16-byte aligned).
//
// Per CTA (one per SM), tiles of 128 samples x 128 inputs of one channel in
// order input block fastest, then channel, then sample block:
//   warp 0        TMA loads of raw tiles into a ring of slots (no per-thread
//                 address arithmetic)
//   warps 1..16   converters, in independent groups that take alternate tiles:
//                 transpose + decode into the group's two plane tiles in
//                 shared memory (128-byte swizzle), conflict-free mapping: a
//                 unit is 4 inputs x 8 samples; (virtual) warp w, lane q takes
//                 inputs 4q .. 4q + 3, sample block b = (w + q) mod 8 and half
//                 h = ((q >> 3) & 1) ^ (w >> 3) -- raw reads hit 32 banks,
//                 8-byte plane writes 16 slots per half-warp
//   one thread    of each group TMA-stores its plane tiles and recycles the
//                 raw slot; a plane buffer is rewritten only after its store
//                 has finished reading shared memory
#include <cstring>

#include "nibble.cuh"
#include "tc_ptx.cuh"
#include "xeng_internal.h"

namespace xeng {
namespace {

constexpr int kDTConvWarps = 16;
constexpr int kDTConvThreads = 32 * kDTConvWarps;
constexpr int kDTThreads = 32 + kDTConvThreads;
constexpr int kDTRaw = 128 * 128;
constexpr int kDTPlane = 128 * 128;
// Pipeline shape, measured on GB300 (full-CHIME decode, 16 GiB in, 32 GiB out):
// one converter group of 16 warps spends its time in the per-tile chain (wait,
// convert, fence, store issue) and reaches 4.2 TB/s whatever the ring depth;
// two groups of 8 warps, each with one plane buffer, and an 8-slot raw ring
// reach 5.5-5.8 TB/s (4 groups: 5.2; two groups with two plane buffers and a
// shallower ring: 5.1-5.4; two CTAs per SM of one group: 4.9).
constexpr int kDTSlots = 8;
constexpr int kDTGroups = 2;
constexpr int kDTPlaneBufs = 1;

// shared memory: a ring of raw tiles, then kP plane-tile pairs per converter group, then the barriers
constexpr size_t dt_smem(int stages, int groups, int pbufs, bool raw = false)
{
    return 1024 + (size_t)stages * kDTRaw + (size_t)groups * pbufs * 2 * kDTPlane + 2 * stages * 8 + 16 +
           (raw ? (size_t)kDTConvWarps * 128 * 8 : 0);
}

struct DecTmaArgs {
    int64_t T;             // samples to decode (t0 .. t0 + T - 1 of the map's block)
    int32_t n_ib, n_tb;    // input blocks, sample blocks per channel
    int64_t n_tiles;
    int32_t N, nf, n_pad;
    int32_t f0;            // first channel of the map's block
    int64_t t0;            // first sample of the map's block
    int *err;
    // batched launches: job j's raw and plane maps are maps[2j], maps[2j + 1]
    const CUtensorMap *maps;
    const DecTmaJob *jobs;
    int32_t n_jobs;
    int2 *partials;        // raw mode: [nf][n_tb][n_pad] per-tile nibble sums (P, Q)
};

// One tile as every role sees it.
struct DtTile {
    const CUtensorMap *rm, *pm;
    int ib, fl, tb, f, N, n_pad, x0;
    int64_t T, t0;
    int2 *part;      // raw-nibble planes: the (P, Q) partial sums of the tile's inputs go to
    int part_row;    // part[part_row * n_pad + input] (null: decoded planes)
};

// Tile order within a block (job): input block fastest, then channel, then
// sample block, so the CTAs working at the same time read neighbouring bytes
// of the same sample rows.  Batched: tiles of job j are tile0[j] ..
// tile0[j + 1] - 1.
template <bool kBatch>
__device__ __forceinline__ DtTile dt_tile(const DecTmaArgs &a, const CUtensorMap *rm, const CUtensorMap *pm,
                                          int64_t tile)
{
    DtTile t;
    if (!kBatch) {
        t.rm = rm;
        t.pm = pm;
        t.ib = (int)(tile % a.n_ib);
        t.fl = (int)((tile / a.n_ib) % a.nf);
        t.tb = (int)(tile / ((int64_t)a.n_ib * a.nf));
        t.f = a.f0 + t.fl;
        t.x0 = 0;
        t.N = a.N;
        t.n_pad = a.n_pad;
        t.T = a.T;
        t.t0 = a.t0;
        t.part = a.partials;
        t.part_row = t.fl * a.n_tb + t.tb;
    } else {
        int lo = 0, hi = a.n_jobs - 1;
        while (lo < hi) {  // last job whose first tile is <= tile
            const int mid = (lo + hi + 1) >> 1;
            if (a.jobs[mid].tile0 <= tile) lo = mid;
            else hi = mid - 1;
        }
        const DecTmaJob &j = a.jobs[lo];
        const int64_t local = tile - j.tile0;
        t.rm = a.maps + 2 * lo;
        t.pm = a.maps + 2 * lo + 1;
        t.ib = (int)(local % j.n_ib);
        t.fl = (int)((local / j.n_ib) % j.F);
        t.tb = (int)(local / ((int64_t)j.n_ib * j.F));
        t.f = t.fl;
        t.x0 = j.x0;
        t.N = j.N;
        t.n_pad = j.n_pad;
        t.T = j.T;
        t.t0 = 0;
        t.part = j.partials;
        t.part_row = t.fl * j.part_n_tb + (j.x0 >> 7) + t.tb;
    }
    return t;
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, uint32_t src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                 ::"l"(map), "r"(x), "r"(y), "r"(src)
                 : "memory");
}

// kRaw: the planes hold the raw nibbles (E4M3 codes of u / 512, see the
// correlator's raw mode) instead of the decoded values, and each tile's
// per-input nibble sums (P, Q) go to a.partials[fl][tb][input].  Batched
// launches (kBatch) decide per job: raw where the job has a partial-sum buffer.
template <int kStages, int kGroups, int kP, bool kBatch, bool kRaw = false>
__global__ void __launch_bounds__(kDTThreads, 1)
decode_tma_kernel(const __grid_constant__ CUtensorMap raw_map, const __grid_constant__ CUtensorMap plane_map,
                  const DecTmaArgs a)
{
    // Each raw slot must belong to one group (kStages a multiple of kGroups):
    // a group waits on a slot's "full" barrier by phase parity, which is only
    // unambiguous if the slot's previous tile was the same group's (then it is
    // consumed, so its load is complete).  A slot shared by groups could still
    // be in an earlier tile's phase of the same parity as awaited.
    static_assert(kDTConvWarps % kGroups == 0 && kStages % kGroups == 0, "groups of whole warps, owning whole slots");
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    uint8_t *sgen = smem_raw + (sbase - raw);
    const uint32_t pbase = sbase + kStages * kDTRaw;                 // plane buffers
    const uint32_t bars = pbase + kGroups * kP * 2 * kDTPlane;
    auto rawf = [&](int s) { return bars + 8u * s; };               // raw tile landed
    auto rawe = [&](int s) { return bars + 8u * (kStages + s); };  // raw tile converted
    // raw mode: per converter warp, partial nibble sums (P, Q) of the tile's 128 inputs
    int2 *scratch = reinterpret_cast<int2 *>(sgen + (bars + 8u * 2 * kStages + 16 - sbase));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *err = a.err;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(rawf(s), 1);
            mbar_init(rawe(s), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!kBatch) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(&raw_map) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(&plane_map) : "memory");
        }
    }
    __syncthreads();

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int stage = 0, issued = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
                const DtTile t = dt_tile<kBatch>(a, &raw_map, &plane_map, tile);
                if (!mbar_try_wait(rawe(stage), phase ^ 1u) &&
                    !mbar_wait(rawe(stage), phase ^ 1u, err, kDevTimeoutProducer)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(rawf(stage), kDTRaw);
                tma_load_3d(sbase + stage * kDTRaw, t.rm, t.ib * 128, t.f, (int)(t.t0 + t.tb * 128), rawf(stage));
                ++issued;
                if (++stage == kStages) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            // whether or not the converters consumed them (they stop early on an
            // error), the last loads must land before the CTA exits: wait for
            // each, bounded in time but not cut short by the error word
            (void)ok;
            for (int k = 1; k <= kStages && k <= issued; k++) {
                int s = stage - k, p = (int)phase;
                if (s < 0) {
                    s += kStages;
                    p ^= 1;
                }
                const uint64_t t_start = globaltimer();
                while (!mbar_try_wait(rawf(s), (uint32_t)p) && globaltimer() - t_start < kWaitLimitNs) {
                }
            }
        }
    } else {
        // ---------------- converters ----------------
        // kGroups independent groups of kGW warps; group g converts the CTA's
        // tiles n = g, g + kGroups, ... (raw slot n mod kStages) into its own
        // kP plane buffers in turn, so several tiles are in conversion at once.
        // Each thread covers the units of kGroups "virtual warps" of the
        // 16-warp mapping.
        constexpr int kGW = kDTConvWarps / kGroups;
        constexpr int kGThreads = 32 * kGW;
        const int cw = warp - 1;
        const int grp = cw / kGW, wl = cw % kGW;
        const int q = lane;  // inputs 4q .. 4q + 3
        const bool storer = wl == 0 && lane == 0;
        const uint32_t bar_a = 1 + 2 * grp, bar_b = 2 + 2 * grp;
        for (int64_t n = grp;; n += kGroups) {
            const int64_t tile = blockIdx.x + n * gridDim.x;
            if (tile >= a.n_tiles) break;
            const DtTile tl = dt_tile<kBatch>(a, &raw_map, &plane_map, tile);
            const int ib = tl.ib, fl = tl.fl, tb = tl.tb;
            const int stage = (int)(n % kStages);
            const uint32_t phase = (uint32_t)((n / kStages) & 1);
            const bool ok = mbar_wait_backoff(rawf(stage), phase, err, kDevTimeoutProducer, XENG_CONV_SLEEP_NS);
            const int pslot = (int)((n / kGroups) % kP);
            const uint32_t pre_s = pbase + (uint32_t)((grp * kP + pslot) * 2 * kDTPlane);
            // the store that last read this plane buffer (the group's kP-th last) is done reading
            if (storer) asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(kP - 1) : "memory");
            // every thread of the group has its raw tile, and the plane buffer is free
            asm volatile("bar.sync %0, %1;" ::"r"(bar_a), "n"(kGThreads) : "memory");
            const uint32_t *rt = reinterpret_cast<const uint32_t *>(sgen + stage * kDTRaw);
            uint8_t *pre = sgen + (pre_s - sbase);
            uint8_t *pim = pre + kDTPlane;
            const int ibase = ib * 128;
            const bool raw = kBatch ? tl.part != nullptr : kRaw;  // uniform over the tile
            uint32_t sp[4] = {0, 0, 0, 0}, sq[4] = {0, 0, 0, 0};  // raw mode: nibble sums of inputs 4q + m
            if (ok) {
                #pragma unroll
                for (int k = 0; k < kGroups; k++) {
                    const int vw = wl + kGW * k;                  // virtual warp 0..15
                    const int b = ((vw & 7) + lane) & 7;          // sample block of this lane
                    const int h = ((lane >> 3) & 1) ^ (vw >> 3);  // which 8 samples of the block
                    const int64_t tbase = (int64_t)tb * 128 + b * 16 + h * 8;  // first sample of the unit
                    uint32_t re[4][2], im[4][2];  // [input m][word g] (samples 4g .. 4g + 3 of the half)
                    #pragma unroll
                    for (int g = 0; g < 2; g++) {
                        uint32_t r[4];
                        #pragma unroll
                        for (int kk = 0; kk < 4; kk++) {
                            const int t = b * 16 + h * 8 + g * 4 + kk;
                            // past the end: value 0 (decoded) or nibbles 0, adding nothing (raw)
                            r[kk] = (tbase + g * 4 + kk < tl.T) ? rt[t * 32 + q] : (raw ? 0u : 0x88888888u);
                        }
                        if (raw) {
                            // transpose, then split: input m's high (Re) and low (Im) nibbles of samples 0..3
                            #pragma unroll
                            for (int m = 0; m < 4; m++) {
                                const uint32_t sel = (uint32_t)m | ((uint32_t)(4 + m) << 4);
                                const uint32_t w =
                                    __byte_perm(__byte_perm(r[0], r[1], sel), __byte_perm(r[2], r[3], sel), 0x5410);
                                re[m][g] = (w >> 4) & 0x0F0F0F0Fu;
                                im[m][g] = w & 0x0F0F0F0Fu;
                                sp[m] = __dp4a(re[m][g], 0x01010101u, sp[m]);
                                sq[m] = __dp4a(im[m][g], 0x01010101u, sq[m]);
                            }
                        } else {
                            // transpose + decode: r[k] byte m = (sample k, input m) -> input m's codes of samples 0..3
                            decode_input4(r, 0, re[0][g], im[0][g]);
                            decode_input4(r, 1, re[1][g], im[1][g]);
                            decode_input4(r, 2, re[2][g], im[2][g]);
                            decode_input4(r, 3, re[3][g], im[3][g]);
                        }
                    }
                    #pragma unroll
                    for (int m = 0; m < 4; m++) {
                        const int i = 4 * q + m;
                        const int off = i * 128 + ((b ^ (i & 7)) << 4) + h * 8;  // row i, chunk b, half h
                        const bool row_ok = ibase + i < tl.N;                    // rows past N are +0.0
                        *reinterpret_cast<uint2 *>(pre + off) =
                            row_ok ? make_uint2(re[m][0], re[m][1]) : make_uint2(0u, 0u);
                        *reinterpret_cast<uint2 *>(pim + off) =
                            row_ok ? make_uint2(im[m][0], im[m][1]) : make_uint2(0u, 0u);
                    }
                }
            }
            if (raw && ok) {
                int4 *sc = reinterpret_cast<int4 *>(scratch + cw * 128 + 4 * q);
                sc[0] = make_int4((int)sp[0], (int)sq[0], (int)sp[1], (int)sq[1]);
                sc[1] = make_int4((int)sp[2], (int)sq[2], (int)sp[3], (int)sq[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // planes visible to the TMA store
            // the second barrier also ORs the group's failure flags, so that all
            // of its threads leave the loop in the same iteration (a named
            // barrier that some threads never reach would not return)
            uint32_t any_fail;
            asm volatile(
                "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
                "bar.red.or.pred p, %2, %3, q;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(any_fail)
                : "r"(ok ? 0u : 1u), "r"(bar_b), "n"(kGThreads)
                : "memory");
            if (storer) {
                if (!any_fail) {
                    const int y = (fl * 2) * tl.n_pad + ib * 128;
                    tma_store_2d(tl.pm, tl.x0 + tb * 128, y, pre_s);
                    tma_store_2d(tl.pm, tl.x0 + tb * 128, y + tl.n_pad, pre_s + kDTPlane);
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                }
                mbar_arrive(rawe(stage));  // the raw slot may be refilled
            }
            if (raw && !any_fail && wl < 4) {
                // the tile's sums of input k = 32 wl + lane over the group's warps (their partials
                // stay until the group's next first barrier, which every reader passes after this)
                const int k = wl * 32 + lane;
                int P = 0, Q = 0;
                #pragma unroll
                for (int w = 0; w < kGW; w++) {
                    const int2 v = scratch[(grp * kGW + w) * 128 + k];
                    P += v.x;
                    Q += v.y;
                }
                tl.part[(int64_t)tl.part_row * tl.n_pad + ibase + k] = make_int2(P, Q);
            }
            if (any_fail) break;
        }
        // every store has finished writing before the CTA exits
        if (storer) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
}

}  // namespace

bool decode_tma_ok(const uint8_t *block, int32_t N)
{
    return N % 16 == 0 && (reinterpret_cast<uintptr_t>(block) & 15) == 0;
}

cudaError_t launch_decode_tma(const uint8_t *block, int64_t T, int32_t F, int32_t N, int32_t f0, int32_t nf,
                              uint8_t *planes, int64_t t_pad, int64_t n_pad, int *err, int num_sms, cudaStream_t s,
                              int2 *partials)
{
    if (nf <= 0 || t_pad <= 0) return cudaSuccess;
    if (!decode_tma_ok(block, N) || T <= 0 || t_pad % 128 != 0 || n_pad % 128 != 0 || t_pad < T || n_pad < N ||
        t_pad > 2147483647LL || (int64_t)nf * 2 * n_pad > 2147483647LL || num_sms <= 0)
        return cudaErrorInvalidValue;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap rm, pm;
    {
        // raw block [T][F][N] bytes: box of 128 inputs x 1 channel x 128 samples; reads past N or T fill 0
        const cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)F, (cuuint64_t)T};
        const cuuint64_t strides[2] = {(cuuint64_t)N, (cuuint64_t)N * F};
        const cuuint32_t box[3] = {128, 1, 128}, estr[3] = {1, 1, 1};
        if (enc(&rm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, (void *)block, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    {
        // planes [nf * 2 * n_pad][t_pad]: box of 128 samples x 128 rows, 128-byte swizzle (the
        // layout the converters write in shared memory)
        const cuuint64_t dims[2] = {(cuuint64_t)t_pad, (cuuint64_t)nf * 2 * n_pad};
        const cuuint64_t strides[1] = {(cuuint64_t)t_pad};
        const cuuint32_t box[2] = {128, 128}, estr[2] = {1, 1};
        if (enc(&pm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void *)planes, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    const bool raw = partials != nullptr;
    auto kern = raw ? decode_tma_kernel<kDTSlots, kDTGroups, kDTPlaneBufs, false, true>
                    : decode_tma_kernel<kDTSlots, kDTGroups, kDTPlaneBufs, false, false>;
    const size_t smem = dt_smem(kDTSlots, kDTGroups, kDTPlaneBufs, raw);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    DecTmaArgs a;
    a.partials = partials;
    a.T = T;
    a.n_ib = (int32_t)(n_pad / 128);
    a.n_tb = (int32_t)(t_pad / 128);
    a.n_tiles = (int64_t)a.n_ib * nf * a.n_tb;
    a.N = N;
    a.nf = nf;
    a.n_pad = (int32_t)n_pad;
    a.f0 = f0;
    a.t0 = 0;
    a.err = err;
    a.maps = nullptr;
    a.jobs = nullptr;
    a.n_jobs = 0;
    const int grid = (int)(a.n_tiles < num_sms ? a.n_tiles : num_sms);
    kern<<<grid, kDTThreads, smem, s>>>(rm, pm, a);
    return cudaGetLastError();
}

namespace {
// sums[fl][i] = sum over the tiles tb of partials[fl][tb][i]
__global__ void plane_sums_kernel(const int2 *__restrict__ partials, int32_t nf, int32_t n_tb, int32_t n_pad,
                                  int2 *__restrict__ sums)
{
    const int64_t total = (int64_t)nf * n_pad;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t fl = k / n_pad, i = k % n_pad;
        const int2 *p = partials + fl * n_tb * n_pad + i;
        int P = 0, Q = 0;
        for (int tb = 0; tb < n_tb; tb++) {
            const int2 v = p[(int64_t)tb * n_pad];
            P += v.x;
            Q += v.y;
        }
        sums[k] = make_int2(P + Q, P - Q);  // (S, D) as the correlator's raw mode uses them
    }
}
}  // namespace

cudaError_t launch_plane_sums(const int2 *partials, int32_t nf, int32_t n_tb, int32_t n_pad, int2 *sums, int num_sms,
                              cudaStream_t s)
{
    if (nf <= 0) return cudaSuccess;
    const int64_t total = (int64_t)nf * n_pad;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 8 * (int64_t)num_sms) blocks = 8 * (int64_t)num_sms;
    plane_sums_kernel<<<(unsigned)blocks, 256, 0, s>>>(partials, nf, n_tb, n_pad, sums);
    return cudaGetLastError();
}

namespace {
// Batched: sums of job j = (S, D) totals over its tile rows of the partials;
// entry k of the launch is job j's (fl, i) with k - jobs[j].first = fl * n_pad + i.
__global__ void plane_sums_batch_kernel(const SumJob *__restrict__ jobs, int32_t n_jobs, int64_t total)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_jobs - 1;
        while (lo < hi) {  // last job whose first entry is <= k
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].first <= k) lo = mid;
            else hi = mid - 1;
        }
        const SumJob &j = jobs[lo];
        const int64_t local = k - j.first;
        const int64_t fl = local / j.n_pad, i = local % j.n_pad;
        const int2 *p = j.partials + fl * j.part_n_tb * j.n_pad + i;
        int P = 0, Q = 0;
        for (int tb = 0; tb < j.n_tb; tb++) {
            const int2 v = p[(int64_t)tb * j.n_pad];
            P += v.x;
            Q += v.y;
        }
        j.sums[local] = make_int2(P + Q, P - Q);
    }
}
}  // namespace

cudaError_t launch_plane_sums_batch(const SumJob *jobs, int32_t n_jobs, int64_t total, int num_sms, cudaStream_t s)
{
    if (n_jobs <= 0 || total <= 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 8 * (int64_t)num_sms) blocks = 8 * (int64_t)num_sms;
    plane_sums_batch_kernel<<<(unsigned)blocks, 256, 0, s>>>(jobs, n_jobs, total);
    return cudaGetLastError();
}

bool encode_decode_tma_maps(const uint8_t *block, int64_t T, int32_t F, int32_t N, uint8_t *planes, int64_t t_pad,
                            int64_t n_pad, CUtensorMap *raw_map, CUtensorMap *plane_map)
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc || !decode_tma_ok(block, N) || t_pad % 128 != 0 || n_pad % 128 != 0 || t_pad > 2147483647LL ||
        (int64_t)F * 2 * n_pad > 2147483647LL || T > 2147483647LL)
        return false;
    const cuuint64_t rdims[3] = {(cuuint64_t)N, (cuuint64_t)F, (cuuint64_t)T};
    const cuuint64_t rstrides[2] = {(cuuint64_t)N, (cuuint64_t)N * F};
    const cuuint32_t rbox[3] = {128, 1, 128}, estr3[3] = {1, 1, 1};
    if (enc(raw_map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, (void *)block, rdims, rstrides, rbox, estr3,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const cuuint64_t pdims[2] = {(cuuint64_t)t_pad, (cuuint64_t)F * 2 * n_pad};
    const cuuint64_t pstrides[1] = {(cuuint64_t)t_pad};
    const cuuint32_t pbox[2] = {128, 128}, estr2[2] = {1, 1};
    return enc(plane_map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void *)planes, pdims, pstrides, pbox, estr2,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Batched launches decide raw or decoded planes per job, so their shared
// memory always has room for the raw mode's partial sums.
cudaError_t prepare_decode_tma_batch()
{
    return cudaFuncSetAttribute(decode_tma_kernel<kDTSlots, kDTGroups, kDTPlaneBufs, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dt_smem(kDTSlots, kDTGroups, kDTPlaneBufs, true));
}

cudaError_t launch_decode_tma_batch(const CUtensorMap *maps, const DecTmaJob *jobs, int n_jobs, int64_t n_tiles,
                                    int *err, int num_sms, cudaStream_t s)
{
    if (n_jobs <= 0 || n_tiles <= 0) return cudaSuccess;
    CUtensorMap unused;
    memset(&unused, 0, sizeof(unused));
    DecTmaArgs a;
    a.partials = nullptr;
    memset(&a, 0, sizeof(a));
    a.n_tiles = n_tiles;
    a.err = err;
    a.maps = maps;
    a.jobs = jobs;
    a.n_jobs = n_jobs;
    const int grid = (int)(n_tiles < num_sms ? n_tiles : num_sms);
    decode_tma_kernel<kDTSlots, kDTGroups, kDTPlaneBufs, true>
        <<<grid, kDTThreads, dt_smem(kDTSlots, kDTGroups, kDTPlaneBufs, true), s>>>(unused, unused, a);
    return cudaGetLastError();
}

}  // namespace xeng
