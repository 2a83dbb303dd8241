// xeng_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>

namespace xeng {

constexpr int kTile = 128;          // inputs per tensor-engine tile, samples per K chunk
constexpr int kMaxChunkSamples = 65536;  // f32 sums stay <= 128 * 65536 = 2^23 (exact)
// Raw-nibble launches (the fused kernel, the tensor path's raw planes): their
// integer sums stay <= 450 * 32768 = 14,745,600 < 2^24, the range in which the
// GPU tests (test_raw_nibble_sums_up_to_2_24, test_raw_nibble_unit_terms_above_2_23)
// show the tensor core's f32 accumulation exact with unit increments.
constexpr int kFusedMaxSamples = 32768;

// Device-side status codes written to the handle's error word.
enum DevStatus : int {
    kDevOk = 0,
    kDevTimeoutProducer = 1,
    kDevTimeoutMma = 2,
    kDevTimeoutEpilogue = 3,
};

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
inline int64_t n_baselines(int64_t n) { return n * (n + 1) / 2; }

// Standalone decode: block [T][F][N] bytes -> planes [nf][2][n_pad][t_pad] E4M3 codes.
cudaError_t launch_decode(const uint8_t *block, int64_t T, int32_t F, int32_t N,
                          int32_t f0, int32_t nf, uint8_t *planes, int64_t t_pad,
                          int64_t n_pad, cudaStream_t s);

// The same decode as a persistent TMA pipeline (one CTA per SM): needs N a
// multiple of 16 and a 16-byte aligned block (decode_tma_ok), t_pad and n_pad
// multiples of 128.  A stalled pipeline sets *err and returns.
bool decode_tma_ok(const uint8_t *block, int32_t N);
// partials non-null: raw-nibble planes (E4M3 codes of u / 512) and per-tile
// per-input nibble sums [nf][t_pad / 128][n_pad] of (P, Q); null: decoded planes.
cudaError_t launch_decode_tma(const uint8_t *block, int64_t T, int32_t F, int32_t N, int32_t f0, int32_t nf,
                              uint8_t *planes, int64_t t_pad, int64_t n_pad, int *err, int num_sms, cudaStream_t s,
                              int2 *partials = nullptr);
// sums[fl][i] = (S, D) = (P + Q, P - Q) over all sample tiles of the partials
cudaError_t launch_plane_sums(const int2 *partials, int32_t nf, int32_t n_tb, int32_t n_pad, int2 *sums, int num_sms,
                              cudaStream_t s);

// Gated / flagged decode of channels [f0, f0 + nf): tile rows are block rows
// idx[0 .. Tg) (one gate's samples); samples whose valid byte is 0 decode to
// zero; usable samples per (channel, input) are added to counts[fl][N] (may be null).
cudaError_t launch_decode_gather(const uint8_t *block, int32_t F, int32_t N, int32_t f0, int32_t nf, const int32_t *idx,
                                 int64_t Tg, const uint8_t *valid, uint8_t *planes, int64_t t_pad, int64_t n_pad,
                                 int32_t *counts, cudaStream_t s);

// Gate accumulator sets of a handle (Sec. IV-C-4) and their usable-sample
// counts: counts[g][k] = (dirty ? counts[g][k] : 0) + base[g] for k < per_gate
// (base: samples of the set pushed without a validity mask).
constexpr int kMaxGates = 64;
struct GateBase {
    int64_t v[kMaxGates];
};
cudaError_t launch_counts_finish(int32_t *counts, int dirty, const GateBase &base, int32_t G, int64_t per_gate,
                                 cudaStream_t s);

// Batched decode: one launch over the tiles of several blocks.
struct DecodeJob {
    const uint8_t *block;  // [T][F][N]
    uint8_t *planes;       // [F][2][n_pad][pitch]: this job fills columns [0, t_pad) of every row
    int64_t T, t_pad, n_pad;
    int64_t pitch;         // bytes between plane rows (>= t_pad)
    int64_t cta0;          // first CTA of this job in the launch
    int32_t F, N;
    int32_t vec_ok;        // 16-byte loads allowed (see decode_vec_ok)
    int32_t pad_;
};
int decode_vec_ok(const uint8_t *block, int32_t N);
// CTAs one job takes in a batched decode launch.
inline int64_t decode_ctas(int64_t t_pad, int64_t n_pad, int64_t F) { return (t_pad / 128) * (n_pad / 128) * F; }
// Time shifting (Sec. IV-C-5): input i of the pushed block is read d_i
// samples late; the samples before the block come from the history.
struct ShiftArgs {
    const int32_t *delay = nullptr;        // [N] delay of input i, samples
    const int32_t *slot = nullptr;         // [N] history column of input i (-1: not delayed)
    const int32_t *chunk_delay = nullptr;  // [ceil(N/16)] delay shared by inputs 16c..16c+15, or -1
    const uint8_t *hist = nullptr;         // [H][F][S] the H samples before the block, delayed inputs only
    int64_t H = 0;
    int32_t S = 0;
};
// Decode samples t0 .. t0 + nt - 1 of the block (T_block samples) with the
// shift applied, channels f0 .. f0 + nf - 1, into planes as launch_decode.
cudaError_t launch_decode_shifted(const uint8_t *block, int64_t t0, int64_t nt, int32_t F, int32_t N, int32_t f0,
                                  int32_t nf, const ShiftArgs &sa, uint8_t *planes, int64_t t_pad, int64_t n_pad,
                                  cudaStream_t s);
// Batched TMA decode: job j's block [T][F][N] into its planes [F][2][n_pad][t_pad]
// through the maps encode_decode_tma_maps writes (device array: raw map 2j,
// plane map 2j + 1); tiles tile0[j] .. tile0[j] + n_ib * F * n_tb - 1 are job
// j's.  prepare_decode_tma_batch sets the kernel's shared-memory limit (call
// it before capturing a launch in a graph).
struct DecTmaJob {
    int64_t tile0;
    int64_t T;
    int32_t n_ib, n_tb, F, N, n_pad;
    int32_t x0;          // first plane column of the job in its plane map (a multiple of 128)
    int2 *partials;      // non-null: raw-nibble planes, the tiles' (P, Q) sums to
                         // partials[fl][x0 / 128 + tb][n_pad] ...
    int32_t part_n_tb;   // ... whose rows per channel are part_n_tb
    int32_t pad_;
};
// Totals of raw-nibble partial sums for several jobs in one launch: job j's
// sums[fl][i] = (S, D) over tile rows 0 .. n_tb - 1 of partials[fl][.][i]
// (rows per channel part_n_tb); its entries are k = first .. first + F * n_pad - 1.
struct SumJob {
    const int2 *partials;
    int2 *sums;
    int64_t first;
    int32_t n_tb, part_n_tb, n_pad, pad_;
};
cudaError_t launch_plane_sums_batch(const SumJob *jobs, int32_t n_jobs, int64_t total, int num_sms, cudaStream_t s);
bool encode_decode_tma_maps(const uint8_t *block, int64_t T, int32_t F, int32_t N, uint8_t *planes, int64_t t_pad,
                            int64_t n_pad, CUtensorMap *raw_map, CUtensorMap *plane_map);
cudaError_t prepare_decode_tma_batch();
cudaError_t launch_decode_tma_batch(const CUtensorMap *maps, const DecTmaJob *jobs, int n_jobs, int64_t n_tiles,
                                    int *err, int num_sms, cudaStream_t s);

// After a plain decode of samples t0 .. t0 + nt - 1 into planes: rewrite the
// rows of the S delayed inputs (inputs[s] has history column s) with their
// shifted samples, as launch_decode_shifted computes them.
cudaError_t launch_shift_fixup(const uint8_t *block, int64_t t0, int64_t nt, int32_t F, int32_t N, int32_t f0,
                               int32_t nf, const ShiftArgs &sa, const int32_t *inputs, uint8_t *planes, int64_t t_pad,
                               int64_t n_pad, cudaStream_t s);
// New history after a block of n samples: the last H samples of (old history,
// block) for the S delayed inputs listed in `inputs`.
cudaError_t launch_shift_history(const uint8_t *hist_old, const uint8_t *block, int64_t n, int32_t F, int32_t N,
                                 const int32_t *inputs, int32_t S, int64_t H, uint8_t *hist_new, cudaStream_t s);

// Decode fused into the correlation for N <= 256 (small_ok: N % 16 == 0, block
// 16-byte aligned): samples t0 .. t0 + nt - 1 (nt <= kFusedMaxSamples) of the
// block (T_block samples), channels f0 .. f0 + nf - 1, stored (accumulate = 0)
// or added into acc [nf][N(N+1)/2][2] (8-byte aligned); no decoded planes.
// Single CTAs over upper-triangle 128 x 128 blocks only (three per channel of
// 129..256 inputs).  The launch's work is split evenly over the CTAs; an item
// cut between CTAs is completed through ws (scratch of small_ws_bytes(num_sms))
// and flags (small_flags_bytes(num_sms), zeroed once: a flag per CTA, the
// count of launches on them and an arrival counter, with which the last CTA of
// each launch advances the count, so replays of a captured launch stay apart).
bool small_ok(const uint8_t *block, int32_t N);
size_t small_ws_bytes(int num_sms);
size_t small_flags_bytes(int num_sms);
cudaError_t launch_correlate_small(const uint8_t *block, int64_t T_block, int64_t t0, int64_t nt, int32_t F, int32_t N,
                                   int32_t f0, int32_t nf, int32_t *acc, int accumulate, int2 *ws, int *flags,
                                   int *err, int num_sms, cudaStream_t s,
                                   const CUtensorMap *maps = nullptr, int32_t spb = 0);
// The raw-block tensor map launch_correlate_small uses (3D: input, channel, sample;
// its stage's box, 128-byte swizzle), and its stage in samples.
cudaError_t encode_small_map(CUtensorMap *map, const uint8_t *block, int64_t T_block, int32_t F, int32_t N);
int small_stage_samples();

// One pass over the raw bytes for N a multiple of 16 up to 4096 (block 16-byte
// aligned; used above 256 inputs): single CTAs over every channel's
// upper-triangle pairs of 128-input blocks, the nibble split and each pair's
// nibble sums in shared memory; nt <= kFusedMaxSamples, acc 8-byte aligned.
bool onepass_ok(const uint8_t *block, int32_t N);
cudaError_t launch_correlate_onepass(const uint8_t *block, int64_t T_block, int64_t t0, int64_t nt, int32_t F,
                                     int32_t N, int32_t f0, int32_t nf, int32_t *acc, int accumulate, int *err,
                                     int num_sms, cudaStream_t s,
                                     const CUtensorMap *maps = nullptr, int32_t spb = 0);
// The raw-block tensor map launch_correlate_onepass uses (3D: input, channel, sample;
// its stage's box, 128-byte swizzle), and its stage in samples.
cudaError_t encode_onepass_map(CUtensorMap *map, const uint8_t *block, int64_t T_block, int32_t F, int32_t N);
int onepass_stage_samples();

// Decode fused into the correlation for 16 <= N <= 4096 (N % 16 == 0, block
// 16-byte aligned), as launch_correlate_small: 2-CTA clusters over every
// channel's upper-triangle pairs of 256-input blocks, nibble sums in shared
// memory; nt <= kFusedMaxSamples, acc 8-byte aligned.
bool pair_ok(const uint8_t *block, int32_t N);
cudaError_t launch_correlate_pair(const uint8_t *block, int64_t T_block, int64_t t0, int64_t nt, int32_t F, int32_t N,
                                  int32_t f0, int32_t nf, int32_t *acc, int accumulate, int *err, int num_sms,
                                  cudaStream_t s,
                                  const CUtensorMap *maps = nullptr, int32_t spb = 0);
// One job of a listed launch of the pair kernel (a batch's jobs in one
// persistent launch): its raw block's tensor map (encode_pair_map, in device
// memory, 64-byte aligned), its output [F][N(N+1)/2][2] (stored) and sizes: nt
// <= kFusedMaxSamples samples in n_k stages, nt2 256-input blocks and
// pairs_per_ch upper-triangle block pairs per channel, its items item0 ..
// item0 + F * pairs_per_ch - 1 of the launch (jobs in increasing item0).
struct PairJob {
    const CUtensorMap *map;
    int32_t *acc;
    int32_t N, nt, n_k, nt2, pairs_per_ch, item0;
};
cudaError_t launch_correlate_pair_listed(const PairJob *jobs, int32_t n_jobs, int64_t n_items, int *err, int num_sms,
                                         cudaStream_t s);
// The raw-block tensor map launch_correlate_pair uses (3D: input, channel, sample;
// its stage's box, 128-byte swizzle), and its stage in samples.
cudaError_t encode_pair_map(CUtensorMap *map, const uint8_t *block, int64_t T_block, int32_t F, int32_t N);
int pair_stage_samples();

// The single-pass kernel (single_pass.cu) that takes a block of N inputs:
// kSingleSmall (N <= 256), kSingleOnepass or kSinglePair (above, by the
// measured cost of their block pairs), or 0 where none applies (N not a
// multiple of 16, block not 16-byte aligned, a kernel switched off, or
// `bounded` and N above the build's XENG_FUSED_MAX_N, where two passes are
// faster).  `force`: 0, a kernel to take for every N it covers, or kSingleNone.
enum SinglePass { kSingleNone = -1, kSingleSmall = 1, kSingleOnepass = 2, kSinglePair = 3 };
// The environment variable XENG_FUSED_KERNEL: "pair", "onepass" (force that
// kernel), "none" (no single pass for the default engine and batches), else 0.
int single_pass_force_from_env();
int single_pass_kernel(const uint8_t *block, int32_t N, int force, bool bounded);
// Scratch of the N <= 256 kernel, allocated at its first launch (flags zeroed
// on the stream) and owned by the caller.
struct SmallScratch {
    int2 *ws = nullptr;
    int *flags = nullptr;
};
cudaError_t small_scratch_alloc(SmallScratch *sc, int num_sms, cudaStream_t s);
void small_scratch_free(SmallScratch *sc);
// One launch of single-pass kernel `kernel` over samples t0 .. t0 + nt - 1
// (nt <= kFusedMaxSamples) and channels f0 .. f0 + nf - 1 of the block.  With
// `maps` (device memory, 64-byte aligned), the samples come instead from
// consecutive blocks of spb stages each, block k through maps[k] (made by
// encode_single_pass_map); block is then unused and t0 must be 0.
cudaError_t launch_single_pass(int kernel, const uint8_t *block, int64_t T_block, int64_t t0, int64_t nt, int32_t F,
                               int32_t N, int32_t f0, int32_t nf, int32_t *acc, int accumulate, SmallScratch *sc,
                               int *err, int num_sms, cudaStream_t s, const CUtensorMap *maps = nullptr,
                               int32_t spb = 0);
// A block's tensor map for `kernel`'s stage tables, and the kernel's stage.
cudaError_t encode_single_pass_map(int kernel, CUtensorMap *map, const uint8_t *block, int64_t T_block, int32_t F,
                                   int32_t N);
int single_pass_stage(int kernel);

// Beamforming (Sec. IV-C-3).  The host fills T, F, N, B, out and err; the
// launcher fills the rest.
struct BfArgs {
    int64_t T = 0;
    int32_t F = 0, N = 0, B = 0;
    int32_t n_kc = 0;       // 128-input K chunks
    int32_t n_tt = 0;       // 128-sample tiles
    int64_t n_items = 0;    // F * n_tt
    int32_t f_fastest = 0;  // item order: channel fastest, else sample tile fastest
    int32_t vec16 = 0;      // B even and out 16-byte aligned: two beams per store
    const uint8_t *block = nullptr;  // [T][F][N]
    int32_t *out = nullptr; // [T][F][B][2]
    const int32_t *corr = nullptr;  // [F][Bp][2] offset terms (8 sum(w_re - w_im), 8 sum(w_re + w_im))
    int *err = nullptr;
};
int beam_padded(int32_t n_beams);  // 4, 8, 16, 32 or 64
cudaError_t launch_beam_weights(const int8_t *w_re, const int8_t *w_im, int32_t F, int32_t B, int32_t N,
                                uint8_t *wdev, int32_t *corr, cudaStream_t s);
cudaError_t launch_beamform(const uint8_t *block, const uint8_t *wdev, const int32_t *corr, BfArgs a, int num_sms,
                            cudaStream_t s);

cudaError_t launch_decode_batch(const DecodeJob *jobs, int n_jobs, int64_t total_ctas, cudaStream_t s);

// Tensor-core correlation of decoded planes (tcgen05, FP8 E4M3, f32 in TMEM).
// acc: int32 [nf][N(N+1)/2][2] of the channel group; accumulate = add to it.
struct TcArgs {
    const uint8_t *planes;
    int64_t t_pad;
    int32_t n_pad;
    int32_t N;
    int32_t nf;
    int32_t *acc;
    int32_t accumulate;
    int32_t *err;
    // raw-nibble planes: per channel of the launch, (S, D) of every input row
    // [nf][n_pad], and the samples integrated (<= kFusedMaxSamples); null: decoded planes
    const int2 *sums = nullptr;
    int64_t n_samples = 0;
};
cudaError_t launch_correlate_tc(const TcArgs &a, int num_sms, cudaStream_t s);
// The same correlation with cta_group::2: clusters of two CTAs compute
// 256 x 256 tiles (a.n_pad must be a multiple of 256).
cudaError_t launch_correlate_tc2(const TcArgs &a, int num_sms, cudaStream_t s);

// Batched (listed) launches: a job table, per-job tensor maps and a work list
// partitioned by CTA, all in device memory.
struct JobDesc {
    int32_t *out;      // [F][N(N+1)/2][2] int32 of the job
    int32_t n_pad;     // inputs rounded up to 128
    int32_t N;
    int32_t mode;      // epilogue: 0 store, 1 add (read-modify-write), 2 atomic add (items share tiles)
    int32_t n_samples; // raw-nibble planes: samples integrated (the offset terms' n)
    const int2 *sums;  // raw-nibble planes: (S, D) per [F][n_pad]; null: decoded planes
};
struct WorkItem {
    int32_t job, fl;   // job index, channel within the job
    int16_t I, J;      // 128-input tile pair, I <= J
    int32_t kc0, kc1;  // 128-sample chunks [kc0, kc1), at most kMaxChunkSamples / 128 of them
};
struct ListArgs {
    const CUtensorMap *maps;   // [n_jobs], 64-byte aligned
    const JobDesc *jobs;       // [n_jobs]
    const WorkItem *items;     // [n_items]
    const int32_t *cta_begin;  // [grid + 1]: CTA b runs items [cta_begin[b], cta_begin[b + 1]);
                               // nullptr: CTA b runs items b, b + grid, b + 2 grid, ... < n_items
    int32_t *err;              // device status word
    int64_t n_items;
};
cudaError_t encode_planes_map(CUtensorMap *map, const uint8_t *planes, int64_t t_pad, int64_t rows);
cudaError_t prepare_correlate_tc_listed();
// Bounded-wait self-test (no fault, no hang): *status = device status word
// after one thread's wait ran out, *left = threads that gave up (all of them).
cudaError_t selftest_wait_timeout(int64_t limit_ns, int *status, int *left);  // kernel attributes; call before any stream capture
cudaError_t launch_correlate_tc_listed(const ListArgs &L, int grid, cudaStream_t s);

// Plain CUDA-core correlation straight from the bytes (dp4a, int32).
cudaError_t launch_correlate_dp4a(const uint8_t *block, int64_t T, int32_t F, int32_t N,
                                  int32_t *acc, int32_t accumulate, cudaStream_t s);

}  // namespace xeng
