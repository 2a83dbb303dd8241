// xeng_api.cu -- the C ABI (include/xeng.h): handle state, argument checks,
// chunking of a push into decode + correlation launches, dumps and counters.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include "../../include/xeng.h"
#include "xeng_internal.h"

using namespace xeng;

static_assert(XENG_MAX_GATES == kMaxGates, "gate set limit of the header and of the kernels");

struct TimedLaunch {
    int kind;  // 0 = decode, 1 = correlate
    cudaEvent_t start, stop;
};

struct xeng_s {
    int32_t N = 0, F = 0;
    int64_t t_integ = 0;
    int32_t engine = XENG_ENGINE_TENSOR;
    int device = 0;
    int num_sms = 0;
    int64_t samples = 0;   // integrated since the last dump
    bool fresh = true;     // accumulators hold nothing yet: the next launch stores
    int32_t *acc = nullptr;        // [F][N(N+1)/2][2]
    uint8_t *planes = nullptr;     // decode buffer of the tensor engine
    int64_t planes_bytes = 0;
    int2 *partials = nullptr;      // raw-nibble planes: per-tile nibble sums [group_f][n_tb][n_pad]
    int2 *sums = nullptr;          // raw-nibble planes: (S, D) per input [group_f][n_pad]
    SmallScratch small;            // single-pass kernel up to 256 inputs: partial blocks of split items,
                                   // the flags that publish them and the launch count
    bool planes_raw = false;       // the last decode wrote raw-nibble planes
    int32_t group_f = 0;           // channels per decode + correlate round
    int64_t chunk_t = 0;           // samples per round
    uint8_t *staging = nullptr;    // device copy of host blocks
    int64_t staging_bytes = 0;
    int *d_err = nullptr;          // device status word of the kernels
    int *h_err = nullptr;          // pinned mirror, refreshed after each push
    int sticky = XENG_OK;
    bool profiling = false;
    xeng_stats_t stats{};
    std::vector<TimedLaunch> timed;
    std::vector<cudaEvent_t> event_pool;
    // host-buffer pipeline: copies in, compute and copies out overlap by channel group
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t ev_start = nullptr, ev_fin = nullptr, ev_in[2] = {nullptr, nullptr}, ev_cmp[2] = {nullptr, nullptr};
    cudaEvent_t ev_sub = nullptr;  // a channel sub-range correlated: its download may start
    uint8_t *pstage[2] = {nullptr, nullptr};
    int64_t pstage_bytes = 0;
    int32_t *gidx = nullptr;       // sample indices of the gates of a gated call
    int64_t gidx_cap = 0;
    // time shifting: delays, history of the delayed inputs (ping-pong), their list
    bool shifted = false;
    int32_t *d_delay = nullptr, *d_slot = nullptr, *d_chunk_delay = nullptr, *d_shift_inputs = nullptr;
    uint8_t *hist[2] = {nullptr, nullptr};
    int hist_cur = 0;
    int64_t hist_H = 0;
    int32_t hist_S = 0;
    bool decode_tma = false;       // decode through the TMA pipeline where the block allows it
    int fused_force = 0;           // single_pass_kernel's force: XENG_FUSED_KERNEL at handle creation
    // gate accumulator sets (xeng_set_gates): acc holds n_gates sets of [F][B][2];
    // set 0's "nothing integrated yet" flag is `fresh`, the others' gate_fresh[g]
    int32_t n_gates = 1;
    std::vector<char> gate_fresh;
    std::vector<int64_t> gate_base;  // per set: samples pushed without a validity mask
    int32_t *counts = nullptr;       // [n_gates][F][N] usable samples of flagged pushes
    bool counts_dirty = false;       // counts hold something since the last dump
};

namespace {

int64_t acc_bytes(const xeng_s *h) { return (int64_t)h->F * n_baselines(h->N) * 8; }

// The decode buffer, allocated on first use.  Synchronizes the device then.
// Build parameter: the tensor path's decode writes raw-nibble planes (E4M3
// codes of u / 512) with per-input nibble sums, and the correlator applies the
// offset in its epilogue (launches of at most kFusedMaxSamples samples); 0:
// decoded planes everywhere.
#ifndef XENG_RAW_PLANES
#define XENG_RAW_PLANES 1
#endif

int64_t planes_rows(int64_t N);

cudaError_t ensure_planes(xeng_s *h)
{
    if (h->planes) return cudaSuccess;
    cudaError_t e = cudaMalloc(&h->planes, (size_t)h->planes_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->planes = nullptr;
        return e;
    }
    if (XENG_RAW_PLANES) {
        // raw-nibble decodes take at most kFusedMaxSamples samples per launch; without
        // the room for their sums every decode writes decoded planes
        const int64_t n_pad = planes_rows(h->N);
        const int64_t n_tb = (h->chunk_t < kFusedMaxSamples ? h->chunk_t : kFusedMaxSamples) / kTile;
        if (cudaMalloc(&h->partials, (size_t)(h->group_f * n_tb * n_pad) * sizeof(int2)) != cudaSuccess ||
            cudaMalloc(&h->sums, (size_t)(h->group_f * n_pad) * sizeof(int2)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(h->partials);
            h->partials = nullptr;
            h->sums = nullptr;
        }
    }
    return cudaSuccess;
}

void free_shift(xeng_s *h)
{
    cudaFree(h->d_delay);
    cudaFree(h->d_slot);
    cudaFree(h->d_chunk_delay);
    cudaFree(h->d_shift_inputs);
    cudaFree(h->hist[0]);
    cudaFree(h->hist[1]);
    h->d_delay = h->d_slot = h->d_chunk_delay = h->d_shift_inputs = nullptr;
    h->hist[0] = h->hist[1] = nullptr;
    h->shifted = false;
    h->hist_H = 0;
    h->hist_S = 0;
    h->hist_cur = 0;
}

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return XENG_OK;
    if (e == cudaErrorMemoryAllocation) return XENG_ERR_NOMEM;
    return XENG_ERR_CUDA;
}

// Surface earlier asynchronous failures: sticky CUDA errors and the kernels'
// device status word (its pinned mirror is written by completed work only).
int check_sticky(xeng_s *h)
{
    if (h->sticky != XENG_OK) return h->sticky;
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->sticky = XENG_ERR_CUDA;
        return h->sticky;
    }
    if (h->h_err && *(volatile int *)h->h_err != 0) {
        h->sticky = XENG_ERR_TIMEOUT;
        return h->sticky;
    }
    return XENG_OK;
}

bool is_device_pointer(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

cudaEvent_t take_event(xeng_s *h)
{
    if (!h->event_pool.empty()) {
        cudaEvent_t e = h->event_pool.back();
        h->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Correlation launches of a handle: one CTA per 128 x 128 tile (default), or
// (build parameter XENG_TC_2CTA=1) cta_group::2 clusters computing 256 x 256
// tiles.  Both give the same bits; the alternative measured no faster on GB300.
#ifndef XENG_TC_2CTA
#define XENG_TC_2CTA 0
#endif
// Channel groups of the host-buffer pipeline.  More groups shorten the ramp at
// either end (the first group's upload and the last group's download overlap
// nothing), but each group's pitched upload copies T rows of (channels x N)
// bytes, and narrow rows cost the copy engine time per row (measured on GB300:
// 207 GB/s at 512 KB rows, 152 at 256 KB, 102 at 128 KB, 212 for a flat copy).
// So the groups are sized for rows of about XENG_PIPE_ROW_BYTES (a build
// parameter), one to eight of them; full CHIME (1024 channels x 2048 inputs)
// gets five (measured: 4 / 5 / 6 / 8 groups -> 130.5 / 128.4 / 133.7 / 144.4 ms
// end to end).
#ifndef XENG_PIPE_ROW_BYTES
#define XENG_PIPE_ROW_BYTES 409600
#endif
// Correlation launches (each followed by its download) per channel group when
// the result goes to host memory.
#ifndef XENG_PIPE_SUBGROUPS
#define XENG_PIPE_SUBGROUPS 4
#endif

// Rows of the decoded planes per channel and plane: N rounded up to the tile.
int64_t planes_rows(int64_t N) { return round_up(N, XENG_TC_2CTA ? 256 : kTile); }

cudaError_t run_correlate(xeng_s *h, TcArgs a, cudaStream_t s)
{
    if (XENG_TC_2CTA) return launch_correlate_tc2(a, h->num_sms, s);
    return launch_correlate_tc(a, h->num_sms, s);
}

// Decode launches of a handle: the persistent TMA pipeline where TMA can
// address the block's rows (N a multiple of 16, 16-byte aligned), else the
// thread-per-row kernel.  Both write the same planes.  The environment variable
// XENG_DECODE_THREADS=1 (read at handle creation) keeps the thread kernel.
#ifndef XENG_DECODE_TMA
#define XENG_DECODE_TMA 1
#endif

cudaError_t run_decode(xeng_s *h, const uint8_t *src, int64_t nt, int32_t F, int32_t N, int32_t f0, int32_t nf,
                       int64_t t_pad, int64_t n_pad, cudaStream_t s)
{
    h->planes_raw = false;
    if (h->decode_tma && decode_tma_ok(src, N)) {
        if (XENG_RAW_PLANES && !XENG_TC_2CTA && h->partials && nt <= kFusedMaxSamples) {
            // raw-nibble planes and their per-input sums (two kernels)
            cudaError_t e = launch_decode_tma(src, nt, F, N, f0, nf, h->planes, t_pad, n_pad, h->d_err, h->num_sms, s,
                                              h->partials);
            if (e == cudaSuccess)
                e = launch_plane_sums(h->partials, nf, (int32_t)(t_pad / kTile), (int32_t)n_pad, h->sums, h->num_sms, s);
            if (e == cudaSuccess) {
                h->planes_raw = true;
                h->stats.launches++;  // the sums kernel
            }
            return e;
        }
        return launch_decode_tma(src, nt, F, N, f0, nf, h->planes, t_pad, n_pad, h->d_err, h->num_sms, s);
    }
    return launch_decode(src, nt, F, N, f0, nf, h->planes, t_pad, n_pad, s);
}

// The tensor engines' single-pass kernels (decode fused into the correlation)
// apply to this block: launches of at most kFusedMaxSamples samples over all
// channels, no planes in HBM.  The default engine takes them up to the build's
// XENG_FUSED_MAX_N inputs, XENG_ENGINE_TENSOR_FUSED for every N they cover.
int fused_kernel(const xeng_s *h, const uint8_t *block)
{
    if (h->engine == XENG_ENGINE_TENSOR) return single_pass_kernel(block, h->N, h->fused_force, true);
    if (h->engine == XENG_ENGINE_TENSOR_FUSED)
        return single_pass_kernel(block, h->N, h->fused_force == kSingleNone ? 0 : h->fused_force, false);
    return 0;
}

bool fused_ok(const xeng_s *h, const uint8_t *block) { return fused_kernel(h, block) != 0; }

cudaError_t launch_fused(xeng_s *h, const uint8_t *block, int64_t T_block, int64_t t0, int64_t nt, int32_t F,
                         int32_t f0, int32_t nf, int32_t *acc, int accumulate, cudaStream_t s)
{
    return launch_single_pass(fused_kernel(h, block), block, T_block, t0, nt, F, h->N, f0, nf, acc, accumulate,
                              &h->small, h->d_err, h->num_sms, s);
}

// Run one kernel launch, bracketed by events when profiling.
template <class F>
cudaError_t timed_launch(xeng_s *h, int kind, cudaStream_t s, F &&fn)
{
    TimedLaunch tl{kind, nullptr, nullptr};
    if (h->profiling) {
        tl.start = take_event(h);
        tl.stop = take_event(h);
        if (tl.start && tl.stop) cudaEventRecord(tl.start, s);
    }
    cudaError_t e = fn();
    if (e != cudaSuccess) return e;
    h->stats.launches++;
    if (kind == 0) h->stats.decode_launches++;
    else h->stats.correlate_launches++;
    if (h->profiling && tl.start && tl.stop) {
        cudaEventRecord(tl.stop, s);
        h->timed.push_back(tl);
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

const char *xeng_strerror(int code)
{
    switch (code) {
    case XENG_OK: return "ok";
    case XENG_ERR_ARG: return "invalid argument";
    case XENG_ERR_RANGE: return "size outside the supported range";
    case XENG_ERR_OVERFLOW: return "push would exceed the integration length";
    case XENG_ERR_NOMEM: return "device allocation failed";
    case XENG_ERR_CUDA: return "CUDA call or kernel failed";
    case XENG_ERR_TIMEOUT: return "device-side wait timed out";
    case XENG_ERR_UNSUPPORTED: return "no usable sm_103 device";
    case XENG_ERR_LATE: return "block of an integration that is already closed";
    default: return "unknown status";
    }
}

int xeng_create(int32_t n_inputs, int32_t n_freq, int64_t t_integ, xeng_t *out_handle)
{
    if (!out_handle) return XENG_ERR_ARG;
    if (n_inputs < 1 || n_inputs > XENG_MAX_INPUTS || n_freq < 1 || t_integ < 1 || t_integ > XENG_MAX_T_INTEG)
        return XENG_ERR_RANGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return XENG_ERR_UNSUPPORTED;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return XENG_ERR_UNSUPPORTED;
    }
    if (prop.major != 10 || prop.minor != 3) return XENG_ERR_UNSUPPORTED;

    xeng_s *h = new (std::nothrow) xeng_s;
    if (!h) return XENG_ERR_NOMEM;
    h->N = n_inputs;
    h->F = n_freq;
    h->t_integ = t_integ;
    h->device = dev;
    h->num_sms = prop.multiProcessorCount;
    {
        const char *env = getenv("XENG_DECODE_THREADS");
        h->decode_tma = XENG_DECODE_TMA && !(env && env[0] == '1');
        h->fused_force = single_pass_force_from_env();
    }

    // Decode buffer: rounds of (group_f channels x chunk_t samples); the
    // budget bounds it at 16 GiB or a quarter of the free memory.  Allocated on
    // first use: handles with up to 256 inputs correlate without it.
    const int64_t n_pad = planes_rows(n_inputs);
    h->chunk_t = round_up(t_integ < kMaxChunkSamples ? t_integ : kMaxChunkSamples, kTile);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    int64_t budget = (int64_t)16 << 30;
    if ((int64_t)free_b / 4 < budget) budget = (int64_t)free_b / 4;
    const int64_t per_ch = 2 * n_pad * h->chunk_t;
    int64_t g = budget / per_ch;
    if (g < 1) g = 1;
    if (g > n_freq) g = n_freq;
    if (g > 65535) g = 65535;
    h->group_f = (int32_t)g;
    h->planes_bytes = g * per_ch;

    cudaError_t e = cudaMalloc(&h->acc, (size_t)acc_bytes(h));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&h->h_err, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        xeng_destroy(h);
        return e == cudaErrorMemoryAllocation ? XENG_ERR_NOMEM : XENG_ERR_CUDA;
    }
    *h->h_err = 0;
    h->gate_fresh.assign(1, 1);
    h->gate_base.assign(1, 0);
    *out_handle = h;
    return XENG_OK;
}

void xeng_destroy(xeng_t h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    cudaFree(h->acc);
    cudaFree(h->planes);
    cudaFree(h->partials);
    cudaFree(h->sums);
    small_scratch_free(&h->small);
    cudaFree(h->staging);
    cudaFree(h->gidx);
    cudaFree(h->counts);
    cudaFree(h->pstage[0]);
    cudaFree(h->pstage[1]);
    if (h->h2d) cudaStreamDestroy(h->h2d);
    if (h->d2h) cudaStreamDestroy(h->d2h);
    for (int k = 0; k < 2; k++) {
        if (h->ev_in[k]) cudaEventDestroy(h->ev_in[k]);
        if (h->ev_cmp[k]) cudaEventDestroy(h->ev_cmp[k]);
    }
    if (h->ev_start) cudaEventDestroy(h->ev_start);
    if (h->ev_fin) cudaEventDestroy(h->ev_fin);
    if (h->ev_sub) cudaEventDestroy(h->ev_sub);
    free_shift(h);
    cudaFree(h->d_err);
    if (h->h_err) cudaFreeHost(h->h_err);
    for (auto &t : h->timed) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    for (auto e : h->event_pool) cudaEventDestroy(e);
    cudaGetLastError();
    delete h;
}

int xeng_set_engine(xeng_t h, int32_t engine)
{
    if (!h) return XENG_ERR_ARG;
    if (engine != XENG_ENGINE_TENSOR && engine != XENG_ENGINE_DP4A && engine != XENG_ENGINE_TENSOR_PLANES &&
        engine != XENG_ENGINE_TENSOR_FUSED)
        return XENG_ERR_ARG;
    if (engine == XENG_ENGINE_DP4A && h->shifted) return XENG_ERR_UNSUPPORTED;
    h->engine = engine;
    return XENG_OK;
}

int xeng_set_delays(xeng_t h, const int32_t *delays)
{
    if (!h) return XENG_ERR_ARG;
    const int32_t N = h->N;
    int32_t H = 0;
    if (delays)
        for (int32_t i = 0; i < N; i++) {
            if (delays[i] < 0 || delays[i] > XENG_MAX_DELAY) return XENG_ERR_RANGE;
            if (delays[i] > H) H = delays[i];
        }
    if (H > 0 && h->engine == XENG_ENGINE_DP4A) return XENG_ERR_UNSUPPORTED;
    cudaDeviceSynchronize();  // queued pushes may still read the old delays and history
    free_shift(h);
    if (H == 0) return cuda_status(cudaGetLastError());
    std::vector<int32_t> slot(N, -1), inputs, chunk((N + 15) / 16, -1);
    for (int32_t i = 0; i < N; i++)
        if (delays[i] > 0) {
            slot[i] = (int32_t)inputs.size();
            inputs.push_back(i);
        }
    for (int32_t c = 0; c * 16 < N; c++) {
        bool same = c * 16 + 16 <= N;
        for (int32_t i = c * 16 + 1; same && i < c * 16 + 16; i++) same = delays[i] == delays[c * 16];
        if (same) chunk[c] = delays[c * 16];
    }
    const int32_t S = (int32_t)inputs.size();
    const int64_t hist_bytes = (int64_t)H * h->F * S;
    cudaError_t e = cudaMalloc(&h->d_delay, sizeof(int32_t) * N);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_slot, sizeof(int32_t) * N);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_chunk_delay, sizeof(int32_t) * chunk.size());
    if (e == cudaSuccess) e = cudaMalloc(&h->d_shift_inputs, sizeof(int32_t) * S);
    if (e == cudaSuccess) e = cudaMalloc(&h->hist[0], (size_t)hist_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&h->hist[1], (size_t)hist_bytes);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_delay, delays, sizeof(int32_t) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_slot, slot.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->d_chunk_delay, chunk.data(), sizeof(int32_t) * chunk.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->d_shift_inputs, inputs.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->hist[0], 0x88, (size_t)hist_bytes);  // value 0 + 0i
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_shift(h);
        return e == cudaErrorMemoryAllocation ? XENG_ERR_NOMEM : XENG_ERR_CUDA;
    }
    h->hist_H = H;
    h->hist_S = S;
    h->shifted = true;
    return XENG_OK;
}

}  // extern "C"

namespace {

// Device copy of a caller block: the block itself, or the staging buffer after
// an asynchronous host-to-device copy on `s`.  Returns nullptr on failure.
const uint8_t *device_block(xeng_s *h, const uint8_t *block, int64_t bytes, cudaStream_t s, int *status)
{
    *status = XENG_OK;
    if (is_device_pointer(block)) return block;
    if (h->staging_bytes < bytes) {
        cudaStreamSynchronize(s);  // queued work may still read the old staging
        cudaFree(h->staging);
        h->staging = nullptr;
        h->staging_bytes = 0;
        if (cudaMalloc(&h->staging, (size_t)bytes) != cudaSuccess) {
            cudaGetLastError();
            *status = XENG_ERR_NOMEM;
            return nullptr;
        }
        h->staging_bytes = bytes;
    }
    cudaError_t e = cudaMemcpyAsync(h->staging, block, (size_t)bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        *status = (h->sticky = cuda_status(e));
        return nullptr;
    }
    return h->staging;
}

// Integrate n samples of the device block into `target` ([F][B][2] int32):
// the first launch stores when `fresh`, every later one adds.  Work is
// ordered after earlier work on `s` and before later work on `s`.
cudaError_t integrate(xeng_s *h, const uint8_t *dblock, int64_t n_samples, int32_t *target, bool fresh,
                      cudaStream_t s, bool apply_shift = false)
{
    const int64_t N = h->N, F = h->F;
    const int64_t n_pad = planes_rows(N);
    const int64_t nb2 = N * (N + 1);
    if (h->engine == XENG_ENGINE_DP4A) {
        return timed_launch(h, 1, s, [&] {
            return launch_correlate_dp4a(dblock, n_samples, (int32_t)F, (int32_t)N, target, fresh ? 0 : 1, s);
        });
    }
    cudaError_t e = cudaSuccess;
    if (!apply_shift && fused_ok(h, dblock)) {
        const int64_t fc = kFusedMaxSamples;
        for (int64_t t0 = 0; t0 < n_samples && e == cudaSuccess; t0 += fc) {
            const int64_t nt = (n_samples - t0) < fc ? (n_samples - t0) : fc;
            const int accumulate = (fresh && t0 == 0) ? 0 : 1;
            e = timed_launch(h, 1, s, [&] {
                return launch_fused(h, dblock, n_samples, t0, nt, (int32_t)F, 0, (int32_t)F, target, accumulate, s);
            });
        }
        return e;
    }
    e = ensure_planes(h);
    for (int64_t t0 = 0; t0 < n_samples && e == cudaSuccess; t0 += h->chunk_t) {
        const int64_t nt = (n_samples - t0) < h->chunk_t ? (n_samples - t0) : h->chunk_t;
        const int64_t t_pad = round_up(nt, kTile);
        const int accumulate = (fresh && t0 == 0) ? 0 : 1;
        for (int64_t f0 = 0; f0 < F && e == cudaSuccess; f0 += h->group_f) {
            const int32_t nf = (int32_t)((F - f0) < h->group_f ? (F - f0) : h->group_f);
            const uint8_t *src = dblock + t0 * F * N;
            if (apply_shift) {
                h->planes_raw = false;  // the fix-up rewrites decoded rows
                ShiftArgs sa;
                sa.delay = h->d_delay;
                sa.slot = h->d_slot;
                sa.chunk_delay = h->d_chunk_delay;
                sa.hist = h->hist[h->hist_cur];
                sa.H = h->hist_H;
                sa.S = h->hist_S;
                e = timed_launch(h, 0, s, [&] {
                    if (h->decode_tma && decode_tma_ok(src, (int32_t)N)) {
                        // plain TMA decode, then the delayed inputs' rows rewritten
                        cudaError_t e2 = launch_decode_tma(src, nt, (int32_t)F, (int32_t)N, (int32_t)f0, nf, h->planes,
                                                           t_pad, n_pad, h->d_err, h->num_sms, s);
                        if (e2 != cudaSuccess) return e2;
                        return launch_shift_fixup(dblock, t0, nt, (int32_t)F, (int32_t)N, (int32_t)f0, nf, sa,
                                                  h->d_shift_inputs, h->planes, t_pad, n_pad, s);
                    }
                    return launch_decode_shifted(dblock, t0, nt, (int32_t)F, (int32_t)N, (int32_t)f0, nf, sa, h->planes,
                                                 t_pad, n_pad, s);
                });
            } else {
                e = timed_launch(h, 0, s, [&] {
                    return run_decode(h, src, nt, (int32_t)F, (int32_t)N, (int32_t)f0, nf, t_pad, n_pad, s);
                });
            }
            if (e != cudaSuccess) break;
            TcArgs a;
            a.planes = h->planes;
            a.t_pad = t_pad;
            a.n_pad = (int32_t)n_pad;
            a.N = (int32_t)N;
            a.nf = nf;
            a.acc = target + f0 * nb2;
            a.accumulate = accumulate;
            a.err = h->d_err;
            a.sums = h->planes_raw ? h->sums : nullptr;
            a.n_samples = nt;
            e = timed_launch(h, 1, s, [&] { return run_correlate(h, a, s); });
        }
    }
    if (e == cudaSuccess && apply_shift) {
        e = launch_shift_history(h->hist[h->hist_cur], dblock, n_samples, (int32_t)F, (int32_t)N, h->d_shift_inputs,
                                 h->hist_S, h->hist_H, h->hist[h->hist_cur ^ 1], s);
        if (e == cudaSuccess) h->hist_cur ^= 1;
    }
    return e;
}

// Streams, events and staging of the host-buffer pipeline (created on first use).
int ensure_pipeline(xeng_s *h, int64_t stage_bytes)
{
    cudaError_t e = cudaSuccess;
    if (!h->h2d) {
        e = cudaStreamCreateWithFlags(&h->h2d, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->d2h, cudaStreamNonBlocking);
        for (int k = 0; k < 2 && e == cudaSuccess; k++) {
            e = cudaEventCreateWithFlags(&h->ev_in[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_cmp[k], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fin, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_sub, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (stage_bytes > h->pstage_bytes) {
        cudaDeviceSynchronize();  // the old staging may still be read by queued work
        cudaFree(h->pstage[0]);
        cudaFree(h->pstage[1]);
        h->pstage[0] = h->pstage[1] = nullptr;
        h->pstage_bytes = 0;
        e = cudaMalloc(&h->pstage[0], (size_t)stage_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&h->pstage[1], (size_t)stage_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return XENG_ERR_NOMEM;
        }
        h->pstage_bytes = stage_bytes;
    }
    return XENG_OK;
}

// One integration of n <= chunk_t samples with the tensor engine, where the
// block (`host_in`) and/or the result (`host_out`) live in host memory: the
// channels are cut into groups; group g's pitched host-to-device copy, its
// decode + correlation and its device-to-host copy run on three streams, so
// transfers of neighbouring groups overlap the compute.  `src` is the block
// (host or device), `target` the device triangle written (store when
// `fresh`, else add).  Returns XENG_OK or an error; host_out is complete when
// `s` passes the point this call enqueues.
int integrate_pipelined(xeng_s *h, const uint8_t *src, bool host_in, int64_t n, int32_t *target, int32_t *host_out,
                        bool fresh, cudaStream_t s)
{
    const int64_t N = h->N, F = h->F;
    const int64_t n_pad = planes_rows(N), t_pad = round_up(n, kTile), nb2 = N * (N + 1);
    int64_t groups = (F * N + XENG_PIPE_ROW_BYTES / 2) / XENG_PIPE_ROW_BYTES;
    groups = groups < 1 ? 1 : groups > 8 ? 8 : groups;
    int64_t pf = (F + groups - 1) / groups;  // channels per group
    if (pf > h->group_f) pf = h->group_f;
    if (pf < 1) pf = 1;
    if (host_in && pf >= F && n >= 2 * kTile) {
        // One channel group (short rows per sample): pipeline over time
        // instead.  Time chunks of the block are contiguous, so each is one flat
        // copy; their correlations add into the int32 triangle (exact in any
        // order), and the download follows the last chunk.
        const int64_t tc = round_up((n + 7) / 8, kTile);
        int st = ensure_pipeline(h, tc * F * N);
        if (st != XENG_OK) return st;
        cudaError_t e = cudaEventRecord(h->ev_start, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->h2d, h->ev_start, 0);
        int k = 0;
        for (int64_t t0 = 0; t0 < n && e == cudaSuccess; t0 += tc, ++k) {
            const int64_t nt = (n - t0) < tc ? (n - t0) : tc;
            const int buf = k & 1;
            if (k >= 2) e = cudaStreamWaitEvent(h->h2d, h->ev_cmp[buf], 0);  // staging reused
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h->pstage[buf], src + t0 * F * N, (size_t)(nt * F * N), cudaMemcpyHostToDevice,
                                    h->h2d);
            if (e == cudaSuccess) e = cudaEventRecord(h->ev_in[buf], h->h2d);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_in[buf], 0);
            if (e == cudaSuccess) e = integrate(h, h->pstage[buf], nt, target, fresh && k == 0, s);
            if (e == cudaSuccess) e = cudaEventRecord(h->ev_cmp[buf], s);
        }
        if (e == cudaSuccess && host_out) {
            e = cudaEventRecord(h->ev_fin, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(h->d2h, h->ev_fin, 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(host_out, target, (size_t)(F * nb2 * 4), cudaMemcpyDeviceToHost, h->d2h);
            if (e == cudaSuccess) e = cudaEventRecord(h->ev_fin, h->d2h);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_fin, 0);
        }
        return cuda_status(e);
    }
    int st = ensure_pipeline(h, host_in ? pf * n * N : 0);
    if (st != XENG_OK) return st;
    cudaError_t e = cudaEventRecord(h->ev_start, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->h2d, h->ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->d2h, h->ev_start, 0);
    int g = 0;
    for (int64_t f0 = 0; f0 < F && e == cudaSuccess; f0 += pf, ++g) {
        const int32_t nf = (int32_t)((F - f0) < pf ? (F - f0) : pf);
        const int buf = g & 1;
        const uint8_t *blk = src;
        int32_t bf = (int32_t)F, bf0 = (int32_t)f0;
        if (host_in) {
            // staging[buf] was last read by the decode of group g - 2, which ev_cmp[buf] follows
            if (g >= 2) e = cudaStreamWaitEvent(h->h2d, h->ev_cmp[buf], 0);
            if (e == cudaSuccess) {
                if (nf == F)  // every channel: the block is contiguous
                    e = cudaMemcpyAsync(h->pstage[buf], src, (size_t)(n * F * N), cudaMemcpyHostToDevice, h->h2d);
                else
                    e = cudaMemcpy2DAsync(h->pstage[buf], (size_t)(nf * N), src + f0 * N, (size_t)(F * N),
                                          (size_t)(nf * N), (size_t)n, cudaMemcpyHostToDevice, h->h2d);
            }
            if (e == cudaSuccess) e = cudaEventRecord(h->ev_in[buf], h->h2d);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_in[buf], 0);
            if (e != cudaSuccess) break;
            blk = h->pstage[buf];
            bf = nf;
            bf0 = 0;
        }
        // Correlation launches per group when the result goes to host memory: each
        // channel sub-range is downloaded as soon as it is done, so the downloads,
        // the bottleneck of a host-to-host step, start a fraction of a group's
        // correlation earlier and end as much sooner after the last one.
        const int32_t subs = host_out ? std::min<int32_t>(XENG_PIPE_SUBGROUPS, nf) : 1;
        const int32_t per = (nf + subs - 1) / subs;
        if (fused_ok(h, blk)) {
            for (int32_t c0 = 0; c0 < nf && e == cudaSuccess; c0 += per) {
                const int32_t nc = std::min<int32_t>(per, nf - c0);
                for (int64_t t0 = 0; t0 < n && e == cudaSuccess; t0 += kFusedMaxSamples) {
                    const int64_t nt = (n - t0) < kFusedMaxSamples ? (n - t0) : kFusedMaxSamples;
                    e = timed_launch(h, 1, s, [&] {
                        return launch_fused(h, blk, n, t0, nt, bf, bf0 + c0, nc, target + (f0 + c0) * nb2,
                                            (fresh && t0 == 0) ? 0 : 1, s);
                    });
                }
                if (e == cudaSuccess && host_out) {
                    e = cudaEventRecord(h->ev_sub, s);
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->d2h, h->ev_sub, 0);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(host_out + (f0 + c0) * nb2, target + (f0 + c0) * nb2,
                                            (size_t)(nc * nb2 * 4), cudaMemcpyDeviceToHost, h->d2h);
                }
            }
            // the last launch was the staging buffer's last reader
            if (e == cudaSuccess) e = cudaEventRecord(h->ev_cmp[buf], s);
            continue;
        }
        e = ensure_planes(h);
        if (e != cudaSuccess) break;
        e = timed_launch(h, 0, s, [&] {
            return run_decode(h, blk, n, bf, (int32_t)N, bf0, nf, t_pad, n_pad, s);
        });
        // the decode was the staging buffer's last reader
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_cmp[buf], s);
        if (e != cudaSuccess) break;
        // the correlation in the same channel sub-ranges, each downloaded as soon as it is done
        for (int32_t c0 = 0; c0 < nf && e == cudaSuccess; c0 += per) {
            const int32_t nc = std::min<int32_t>(per, nf - c0);
            TcArgs a;
            a.planes = h->planes + (int64_t)c0 * 2 * n_pad * t_pad;
            a.t_pad = t_pad;
            a.n_pad = (int32_t)n_pad;
            a.N = (int32_t)N;
            a.nf = nc;
            a.acc = target + (f0 + c0) * nb2;
            a.accumulate = fresh ? 0 : 1;
            a.err = h->d_err;
            a.sums = h->planes_raw ? h->sums + (int64_t)c0 * n_pad : nullptr;
            a.n_samples = n;
            e = timed_launch(h, 1, s, [&] { return run_correlate(h, a, s); });
            if (e == cudaSuccess && host_out) {
                e = cudaEventRecord(h->ev_sub, s);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(h->d2h, h->ev_sub, 0);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(host_out + (f0 + c0) * nb2, target + (f0 + c0) * nb2, (size_t)(nc * nb2 * 4),
                                        cudaMemcpyDeviceToHost, h->d2h);
            }
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_fin, host_out ? h->d2h : s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_fin, 0);
    return cuda_status(e);
}

}  // namespace

extern "C" {

int xeng_push(xeng_t h, const uint8_t *block, int64_t n_samples, void *stream)
{
    if (!h) return XENG_ERR_ARG;
    if (n_samples < 0) return XENG_ERR_ARG;
    if (n_samples > 0 && !block) return XENG_ERR_ARG;
    int st = check_sticky(h);
    if (st != XENG_OK) return st;
    if (h->n_gates > 1) return XENG_ERR_ARG;  // several gate sets: xeng_push_gated names the set
    if (h->samples + n_samples > h->t_integ) return XENG_ERR_OVERFLOW;
    if (n_samples == 0) return XENG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (h->engine != XENG_ENGINE_DP4A && n_samples <= h->chunk_t && !is_device_pointer(block) && !h->shifted) {
        st = integrate_pipelined(h, block, true, n_samples, h->acc, nullptr, h->fresh, s);
        if (st != XENG_OK) return (h->sticky = st);
    } else {
        const uint8_t *dblock = device_block(h, block, n_samples * h->F * h->N, s, &st);
        if (!dblock) return st;
        cudaError_t e = integrate(h, dblock, n_samples, h->acc, h->fresh, s, h->shifted);
        if (e != cudaSuccess) return (h->sticky = cuda_status(e));
    }
    cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    h->samples += n_samples;
    h->fresh = false;
    h->gate_base[0] += n_samples;  // every input of every sample usable
    return XENG_OK;
}

int xeng_correlate(xeng_t h, const uint8_t *block, int64_t n_samples, int32_t *out, void *stream)
{
    if (!h || !out) return XENG_ERR_ARG;
    if (n_samples < 0 || (n_samples > 0 && !block)) return XENG_ERR_ARG;
    int st = check_sticky(h);
    if (st != XENG_OK) return st;
    if (n_samples > h->t_integ) return XENG_ERR_OVERFLOW;
    if (h->shifted) return XENG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    const bool dev_out = is_device_pointer(out);
    if (!dev_out && (h->samples > 0 || !h->fresh)) return XENG_ERR_ARG;  // would clobber an open integration
    if (dev_out && (reinterpret_cast<uintptr_t>(out) & 7) != 0) return XENG_ERR_ARG;  // kernels store (Re, Im) pairs
    const int64_t bytes = acc_bytes(h);
    cudaError_t e = cudaSuccess;
    if (n_samples == 0) {
        if (dev_out) return cuda_status(cudaMemsetAsync(out, 0, (size_t)bytes, s));
        e = cudaStreamSynchronize(s);
        memset(out, 0, (size_t)bytes);
        return cuda_status(e);
    }
    const bool dev_in = is_device_pointer(block);
    if (h->engine != XENG_ENGINE_DP4A && n_samples <= h->chunk_t && (!dev_in || !dev_out)) {
        // host buffers: copies overlap the compute, group by group
        st = integrate_pipelined(h, block, !dev_in, n_samples, dev_out ? out : h->acc, dev_out ? nullptr : out, true, s);
        if (st == XENG_OK) e = cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (st == XENG_OK && e == cudaSuccess && !dev_out) e = cudaStreamSynchronize(s);
        if (st != XENG_OK) return (h->sticky = st);
        if (e != cudaSuccess) return (h->sticky = cuda_status(e));
        return dev_out ? XENG_OK : check_sticky(h);
    }
    const uint8_t *dblock = device_block(h, block, n_samples * h->F * h->N, s, &st);
    if (!dblock) return st;
    // device output: written in place; host output: through the accumulators
    e = integrate(h, dblock, n_samples, dev_out ? out : h->acc, true, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && !dev_out) {
        e = cudaMemcpyAsync(out, h->acc, (size_t)bytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) return (h->sticky = cuda_status(e));
    return dev_out ? XENG_OK : check_sticky(h);
}

int xeng_correlate_gated(xeng_t h, const uint8_t *block, int64_t n_samples, const int32_t *gate, int32_t n_gates,
                         const uint8_t *valid, int32_t *out, int32_t *counts, void *stream)
{
    if (!h || !gate || !out || n_gates < 1 || n_samples < 0 || (n_samples > 0 && !block)) return XENG_ERR_ARG;
    int st = check_sticky(h);
    if (st != XENG_OK) return st;
    if (n_samples > h->t_integ) return XENG_ERR_OVERFLOW;
    if (n_samples > h->chunk_t) return XENG_ERR_RANGE;
    if (h->engine == XENG_ENGINE_DP4A) return XENG_ERR_ARG;
    if (h->shifted) return XENG_ERR_UNSUPPORTED;
    if (!is_device_pointer(out) || (counts && !is_device_pointer(counts)) || (valid && !is_device_pointer(valid)) ||
        (n_samples > 0 && !is_device_pointer(block)) || (reinterpret_cast<uintptr_t>(out) & 7) != 0)
        return XENG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = h->N, F = h->F;
    const int64_t n_pad = planes_rows(N), nb2 = N * (N + 1);
    // the samples of each gate, in time order
    std::vector<int64_t> cnt(n_gates + 1, 0);
    for (int64_t t = 0; t < n_samples; t++)
        if (gate[t] >= 0 && gate[t] < n_gates) cnt[gate[t] + 1]++;
    for (int g = 0; g < n_gates; g++) cnt[g + 1] += cnt[g];
    std::vector<int32_t> idx((size_t)std::max<int64_t>(cnt[n_gates], 1));
    {
        std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
        for (int64_t t = 0; t < n_samples; t++)
            if (gate[t] >= 0 && gate[t] < n_gates) idx[fill[gate[t]]++] = (int32_t)t;
    }
    cudaError_t e = cudaSuccess;
    if ((int64_t)idx.size() > h->gidx_cap) {
        e = cudaStreamSynchronize(s);  // an earlier gated call may still read the old list
        cudaFree(h->gidx);
        h->gidx = nullptr;
        h->gidx_cap = 0;
        if (e == cudaSuccess) e = cudaMalloc(&h->gidx, idx.size() * sizeof(int32_t));
        if (e != cudaSuccess) return (h->sticky = cuda_status(e));
        h->gidx_cap = (int64_t)idx.size();
    }
    e = ensure_planes(h);
    if (e != cudaSuccess) return (h->sticky = cuda_status(e));
    e = cudaMemcpyAsync(h->gidx, idx.data(), idx.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // idx is pageable and goes out of scope
    if (e == cudaSuccess && counts) e = cudaMemsetAsync(counts, 0, (size_t)(n_gates * F * N * 4), s);
    for (int g = 0; g < n_gates && e == cudaSuccess; g++) {
        const int64_t Tg = cnt[g + 1] - cnt[g];
        int32_t *out_g = out + (int64_t)g * F * nb2;
        if (Tg == 0) {
            e = cudaMemsetAsync(out_g, 0, (size_t)(F * nb2 * 4), s);
            continue;
        }
        const int64_t t_pad = round_up(Tg, kTile);
        for (int64_t f0 = 0; f0 < F && e == cudaSuccess; f0 += h->group_f) {
            const int32_t nf = (int32_t)((F - f0) < h->group_f ? (F - f0) : h->group_f);
            e = timed_launch(h, 0, s, [&] {
                return launch_decode_gather(block, (int32_t)F, (int32_t)N, (int32_t)f0, nf, h->gidx + cnt[g], Tg, valid,
                                            h->planes, t_pad, n_pad,
                                            counts ? counts + ((int64_t)g * F + f0) * N : nullptr, s);
            });
            if (e != cudaSuccess) break;
            TcArgs a;
            a.planes = h->planes;
            a.t_pad = t_pad;
            a.n_pad = (int32_t)n_pad;
            a.N = (int32_t)N;
            a.nf = nf;
            a.acc = out_g + f0 * nb2;
            a.accumulate = 0;
            a.err = h->d_err;
            e = timed_launch(h, 1, s, [&] { return run_correlate(h, a, s); });
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return (h->sticky = cuda_status(e));
    return XENG_OK;
}

namespace {
// Gate set g holds nothing of the current integration (its next launch stores).
bool set_fresh(const xeng_s *h, int g) { return g == 0 ? h->fresh : h->gate_fresh[g] != 0; }
void mark_set_used(xeng_s *h, int g)
{
    if (g == 0) h->fresh = false;
    else h->gate_fresh[g] = 0;
}

// Start a new integration on every gate set.
cudaError_t reset_integration(xeng_s *h, cudaStream_t s)
{
    h->samples = 0;
    h->fresh = true;
    std::fill(h->gate_fresh.begin(), h->gate_fresh.end(), 1);
    std::fill(h->gate_base.begin(), h->gate_base.end(), 0);
    cudaError_t e = cudaSuccess;
    if (h->counts_dirty) e = cudaMemsetAsync(h->counts, 0, (size_t)h->n_gates * h->F * h->N * 4, s);
    h->counts_dirty = false;
    return e;
}
}  // namespace

int64_t xeng_dump(xeng_t h, int32_t *out, void *stream)
{
    if (!h || !out) return XENG_ERR_ARG;
    int st = check_sticky(h);
    if (st != XENG_OK) return st;
    if (h->n_gates > 1) return XENG_ERR_ARG;  // several gate sets: xeng_dump_gated
    cudaStream_t s = (cudaStream_t)stream;
    const bool dev_out = is_device_pointer(out);
    const int64_t bytes = acc_bytes(h);
    cudaError_t e;
    if (h->fresh) {
        if (dev_out) {
            e = cudaMemsetAsync(out, 0, (size_t)bytes, s);
        } else {
            e = cudaStreamSynchronize(s);
            memset(out, 0, (size_t)bytes);
        }
    } else {
        e = cudaMemcpyAsync(out, h->acc, (size_t)bytes, dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && !dev_out) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) return (h->sticky = cuda_status(e));
    if (!dev_out) {
        st = check_sticky(h);
        if (st != XENG_OK) return st;
    }
    const int64_t n = h->samples;
    e = reset_integration(h, s);
    if (e != cudaSuccess) return (h->sticky = cuda_status(e));
    return n;
}

int xeng_set_gates(xeng_t h, int32_t n_gates)
{
    if (!h) return XENG_ERR_ARG;
    if (n_gates < 1 || n_gates > XENG_MAX_GATES) return XENG_ERR_RANGE;
    int st = check_sticky(h);
    if (st != XENG_OK) return st;
    if (h->samples > 0 || !h->fresh) return XENG_ERR_ARG;  // an integration is in progress
    cudaError_t e = cudaDeviceSynchronize();  // queued work may still use the old sets
    if (e != cudaSuccess) return (h->sticky = cuda_status(e));
    const size_t counts_bytes = (size_t)n_gates * h->F * h->N * 4;
    if (n_gates != h->n_gates) {
        cudaFree(h->acc);
        h->acc = nullptr;
        e = cudaMalloc(&h->acc, (size_t)n_gates * acc_bytes(h));
        if (e != cudaSuccess) {
            // keep the handle usable with one set
            cudaGetLastError();
            h->n_gates = 1;
            if (cudaMalloc(&h->acc, (size_t)acc_bytes(h)) != cudaSuccess) {
                cudaGetLastError();
                h->acc = nullptr;
                h->sticky = XENG_ERR_NOMEM;
            }
            cudaFree(h->counts);
            h->counts = nullptr;
            h->gate_fresh.assign(1, 1);
            h->gate_base.assign(1, 0);
            return XENG_ERR_NOMEM;
        }
        cudaFree(h->counts);
        h->counts = nullptr;
    }
    if (!h->counts) {
        e = cudaMalloc(&h->counts, counts_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->counts = nullptr;
            return XENG_ERR_NOMEM;
        }
    }
    e = cudaMemset(h->counts, 0, counts_bytes);
    if (e != cudaSuccess) return (h->sticky = cuda_status(e));
    h->n_gates = n_gates;
    h->gate_fresh.assign(n_gates, 1);
    h->gate_base.assign(n_gates, 0);
    h->counts_dirty = false;
    h->fresh = true;
    return XENG_OK;
}

int xeng_push_gated(xeng_t h, const uint8_t *block, int64_t n_samples, const int32_t *gate, const uint8_t *valid,
                    void *stream)
{
    if (!h || n_samples < 0 || (n_samples > 0 && !block)) return XENG_ERR_ARG;
    int st = check_sticky(h);
    if (st != XENG_OK) return st;
    if (h->samples + n_samples > h->t_integ) return XENG_ERR_OVERFLOW;
    if (h->engine == XENG_ENGINE_DP4A) return XENG_ERR_ARG;
    if (h->shifted) return XENG_ERR_UNSUPPORTED;
    if (n_samples == 0) return XENG_OK;
    if (!is_device_pointer(block) || (valid && !is_device_pointer(valid))) return XENG_ERR_ARG;
    if (valid && !h->counts) {
        cudaError_t e = cudaMalloc(&h->counts, (size_t)h->n_gates * h->F * h->N * 4);
        if (e == cudaSuccess) e = cudaMemset(h->counts, 0, (size_t)h->n_gates * h->F * h->N * 4);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFree(h->counts);
            h->counts = nullptr;
            return XENG_ERR_NOMEM;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t G = h->n_gates;
    const int64_t N = h->N, F = h->F;
    const int64_t n_pad = planes_rows(N), nb2 = N * (N + 1);
    // the samples of each set, in time order (rows of the block)
    std::vector<int64_t> cnt(G + 1, 0);
    for (int64_t t = 0; t < n_samples; t++) {
        const int32_t g = gate ? gate[t] : 0;
        if (g >= 0 && g < G) cnt[g + 1]++;
    }
    for (int g = 0; g < G; g++) cnt[g + 1] += cnt[g];
    std::vector<int32_t> idx((size_t)std::max<int64_t>(cnt[G], 1));
    {
        std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
        for (int64_t t = 0; t < n_samples; t++) {
            const int32_t g = gate ? gate[t] : 0;
            if (g >= 0 && g < G) idx[fill[g]++] = (int32_t)t;
        }
    }
    cudaError_t e = cudaSuccess;
    if ((int64_t)idx.size() > h->gidx_cap) {
        e = cudaStreamSynchronize(s);  // an earlier gated call may still read the old list
        cudaFree(h->gidx);
        h->gidx = nullptr;
        h->gidx_cap = 0;
        if (e == cudaSuccess) e = cudaMalloc(&h->gidx, idx.size() * sizeof(int32_t));
        if (e != cudaSuccess) return (h->sticky = cuda_status(e));
        h->gidx_cap = (int64_t)idx.size();
    }
    e = ensure_planes(h);
    // the list is rewritten by the next gated call: this call's launches read it first
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->gidx, idx.data(), idx.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // idx is pageable and goes out of scope
    for (int g = 0; g < G && e == cudaSuccess; g++) {
        const int64_t Tg = cnt[g + 1] - cnt[g];
        if (Tg == 0) continue;
        int32_t *set = h->acc + (int64_t)g * F * nb2;
        // rounds of at most chunk_t samples of the set: exact f32 sums per launch
        for (int64_t k0 = 0; k0 < Tg && e == cudaSuccess; k0 += h->chunk_t) {
            const int64_t nk = std::min<int64_t>(h->chunk_t, Tg - k0);
            const int64_t t_pad = round_up(nk, kTile);
            for (int64_t f0 = 0; f0 < F && e == cudaSuccess; f0 += h->group_f) {
                const int32_t nf = (int32_t)((F - f0) < h->group_f ? (F - f0) : h->group_f);
                e = timed_launch(h, 0, s, [&] {
                    return launch_decode_gather(block, (int32_t)F, (int32_t)N, (int32_t)f0, nf, h->gidx + cnt[g] + k0,
                                                nk, valid, h->planes, t_pad, n_pad,
                                                valid ? h->counts + ((int64_t)g * F + f0) * N : nullptr, s);
                });
                if (e != cudaSuccess) break;
                TcArgs a;
                a.planes = h->planes;
                a.t_pad = t_pad;
                a.n_pad = (int32_t)n_pad;
                a.N = (int32_t)N;
                a.nf = nf;
                a.acc = set + f0 * nb2;
                a.accumulate = set_fresh(h, g) ? 0 : 1;
                a.err = h->d_err;
                e = timed_launch(h, 1, s, [&] { return run_correlate(h, a, s); });
            }
            mark_set_used(h, g);
        }
        if (valid) h->counts_dirty = true;
        else h->gate_base[g] += Tg;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return (h->sticky = cuda_status(e));
    h->samples += n_samples;
    return XENG_OK;
}

int64_t xeng_dump_gated(xeng_t h, int32_t *out, int32_t *counts, void *stream)
{
    if (!h || !out) return XENG_ERR_ARG;
    int st = check_sticky(h);
    if (st != XENG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const bool dev_out = is_device_pointer(out);
    const bool dev_counts = counts && is_device_pointer(counts);
    if (dev_out && (reinterpret_cast<uintptr_t>(out) & 3) != 0) return XENG_ERR_ARG;
    const int32_t G = h->n_gates;
    const int64_t set_bytes = acc_bytes(h);
    const int64_t counts_bytes = (int64_t)G * h->F * h->N * 4;
    cudaError_t e = cudaSuccess;
    if (!dev_out || (counts && !dev_counts)) e = cudaStreamSynchronize(s);  // host memory is written below
    for (int g = 0; g < G && e == cudaSuccess; g++) {
        const bool fresh = set_fresh(h, g);
        int32_t *dst = out + (int64_t)g * (set_bytes / 4);
        if (fresh) {
            if (dev_out) e = cudaMemsetAsync(dst, 0, (size_t)set_bytes, s);
            else memset(dst, 0, (size_t)set_bytes);
        } else {
            e = cudaMemcpyAsync(dst, h->acc + (int64_t)g * (set_bytes / 4), (size_t)set_bytes,
                                dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
        }
    }
    if (e == cudaSuccess && counts) {
        if (!h->counts) {
            e = cudaMalloc(&h->counts, (size_t)counts_bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                h->counts = nullptr;
                return XENG_ERR_NOMEM;
            }
            h->counts_dirty = false;
        }
        GateBase base;
        for (int g = 0; g < kMaxGates; g++) base.v[g] = g < G ? h->gate_base[g] : 0;
        e = launch_counts_finish(h->counts, h->counts_dirty ? 1 : 0, base, G, (int64_t)h->F * h->N, s);
        h->counts_dirty = true;  // the buffer now holds this integration's counts: cleared below
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(counts, h->counts, (size_t)counts_bytes,
                                dev_counts ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    }
    const int64_t n = h->samples;
    if (e == cudaSuccess) e = reset_integration(h, s);
    if (e == cudaSuccess && (!dev_out || (counts && !dev_counts))) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return (h->sticky = cuda_status(e));
    if (!dev_out || (counts && !dev_counts)) {
        st = check_sticky(h);
        if (st != XENG_OK) return st;
    }
    return n;
}

int xeng_decode(const uint8_t *block, int64_t n_samples, int32_t n_freq, int32_t n_inputs, int32_t f0, int32_t nf,
                uint8_t *planes, void *stream)
{
    if (!block || !planes) return XENG_ERR_ARG;
    if (n_samples < 1 || n_inputs < 1 || n_inputs > XENG_MAX_INPUTS || n_freq < 1 || f0 < 0 || nf < 1 ||
        f0 + nf > n_freq || nf > 65535 || n_samples > XENG_MAX_T_INTEG)
        return XENG_ERR_RANGE;
    if (!is_device_pointer(block) || !is_device_pointer(planes)) return XENG_ERR_ARG;
    const int64_t t_pad = round_up(n_samples, kTile);
    const int64_t n_pad = round_up(n_inputs, kTile);
    if (t_pad / kTile > 2147483647LL) return XENG_ERR_RANGE;
    cudaStream_t s = (cudaStream_t)stream;
    if (!decode_tma_ok(block, n_inputs)) return cuda_status(launch_decode(block, n_samples, n_freq, n_inputs, f0, nf,
                                                                          planes, t_pad, n_pad, s));
    // the TMA pipeline: its status word lives on the stream for this call only
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int *d_status = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&d_status), sizeof(int), s);
    if (e != cudaSuccess) return cuda_status(e);
    int h_status = 0;
    e = cudaMemsetAsync(d_status, 0, sizeof(int), s);
    if (e == cudaSuccess)
        e = launch_decode_tma(block, n_samples, n_freq, n_inputs, f0, nf, planes, t_pad, n_pad, d_status, sms, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    const cudaError_t ef = cudaFreeAsync(d_status, s);
    if (e == cudaSuccess) e = ef;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    return h_status != 0 ? XENG_ERR_TIMEOUT : XENG_OK;
}

int xeng_selftest_wait_timeout(int64_t limit_ns, int32_t *status, int32_t *threads_left)
{
    if (!status || !threads_left || limit_ns < 0 || limit_ns > 1000000000LL) return XENG_ERR_ARG;
    int st = 0, left = 0;
    cudaError_t e = selftest_wait_timeout(limit_ns, &st, &left);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return XENG_ERR_CUDA;
    }
    *status = st;
    *threads_left = left;
    return XENG_OK;
}

int xeng_set_profiling(xeng_t h, int32_t on)
{
    if (!h) return XENG_ERR_ARG;
    h->profiling = on != 0;
    return XENG_OK;
}

int xeng_get_stats(xeng_t h, xeng_stats_t *stats, int32_t reset)
{
    if (!h || !stats) return XENG_ERR_ARG;
    for (auto &t : h->timed) {
        float ms = 0.f;
        if (cudaEventSynchronize(t.stop) == cudaSuccess && cudaEventElapsedTime(&ms, t.start, t.stop) == cudaSuccess) {
            if (t.kind == 0) {
                h->stats.decode_ms += ms;
                h->stats.timed_decode++;
            } else {
                h->stats.correlate_ms += ms;
                h->stats.timed_correlate++;
            }
        }
        h->event_pool.push_back(t.start);
        h->event_pool.push_back(t.stop);
    }
    h->timed.clear();
    *stats = h->stats;
    if (reset) h->stats = xeng_stats_t{};
    return check_sticky(h);
}

}  // extern "C"
