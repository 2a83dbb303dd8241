/*
 * xeng.h -- C ABI of the GB300 correlator X-engine (libxeng.so).
 *
 * The operation (paper Sec. IV-C-1 "Full Correlation", cost in Eq. 1): for
 * every frequency channel f and every input pair i <= j, integrate the
 * visibility
 *
 *     V_ij(f) = sum_t x_i(t, f) * conj(x_j(t, f))
 *
 * over all N(N+1)/2 pairs (autocorrelations included) and over every sample
 * pushed since the last dump.  Samples are 4+4-bit offset-encoded complex
 * numbers (Sec. II-A and its footnote: each nibble stores value + 8, values
 * in [-8, 7]); the high nibble is the real part, the low nibble the
 * imaginary part.  The arithmetic is exact: results are bit-identical to an
 * integer reference for every input.
 *
 * Layouts
 *   block  uint8  [n_samples][n_freq][n_inputs]   (input index fastest)
 *   out    int32  [n_freq][N(N+1)/2][2]           (Re, Im) pairs, per channel
 *          the upper triangle row-major: pair (i, j), i <= j, sits at
 *          i*N - i*(i-1)/2 + (j - i).
 *
 * Conventions
 *   - Every entry point returns XENG_OK (0) or a negative XENG_ERR_* code
 *     (xeng_dump returns the number of integrated samples on success); none
 *     aborts or prints.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued on it asynchronously unless stated.
 *   - Asynchronous CUDA faults and device-side wait time-outs are reported
 *     as XENG_ERR_CUDA / XENG_ERR_TIMEOUT by the next call on the handle and
 *     stay sticky for that handle.
 *   - A handle is not thread-safe: one thread drives it at a time.
 *   - The library owns all device state of a handle; the caller owns every
 *     buffer passed in.
 *   - The library needs an sm_103 (GB300-class) device; on anything else
 *     xeng_create returns XENG_ERR_UNSUPPORTED.  There is no CPU fallback.
 */
#ifndef XENG_H
#define XENG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define XENG_API __attribute__((visibility("default")))

/* Status codes. */
#define XENG_OK               0
#define XENG_ERR_ARG         -1  /* NULL handle/pointer or invalid value      */
#define XENG_ERR_RANGE       -2  /* size outside the supported range          */
#define XENG_ERR_OVERFLOW    -3  /* push would integrate more than t_integ    */
#define XENG_ERR_NOMEM       -4  /* device allocation failed                  */
#define XENG_ERR_CUDA        -5  /* a CUDA call or kernel failed              */
#define XENG_ERR_TIMEOUT     -6  /* a device-side wait gave up (kernel status) */
#define XENG_ERR_UNSUPPORTED -7  /* no usable sm_103 device                    */
#define XENG_ERR_LATE        -8  /* serving: block of an integration already closed */

/* Limits.  t_integ <= 2^24 - 1 keeps every |Re|, |Im| <= 128 * t_integ below
 * 2^31, so the int32 result of an integration cannot overflow (per sample
 * Re lies in [-112, 128] and |Im| <= 120). */
#define XENG_MAX_INPUTS   4096
#define XENG_MAX_T_INTEG  16777215LL

/* Correlation engines (all give identical bits). */
#define XENG_ENGINE_TENSOR        0  /* tcgen05 tensor cores (default): for N <= 3584 a multiple of 16 (block
                                        16-byte aligned) one kernel splits the raw bytes in shared memory and
                                        correlates them -- N <= 256: single CTAs over 128-input blocks
                                        (scratch of 256 KB per SM, allocated at the first such call); above:
                                        single CTAs over 128-input block pairs or 2-CTA clusters over
                                        256-input block pairs, whichever does less padded work for N.  The
                                        environment variable XENG_FUSED_KERNEL=onepass or =pair (read by
                                        xeng_create) forces one of the two for every such N.  Otherwise as
                                        XENG_ENGINE_TENSOR_PLANES                                            */
#define XENG_ENGINE_DP4A          1  /* plain CUDA-core kernel: int8 dp4a straight from the bytes            */
#define XENG_ENGINE_TENSOR_PLANES 2  /* two passes: decode to FP8 planes in HBM, then the tensor-core GEMM
                                        (decode buffer of up to 16 GiB, allocated at the first such call)    */
#define XENG_ENGINE_TENSOR_FUSED  3  /* the default engine's single pass for every N that is a multiple of
                                        16 (block 16-byte aligned), also above the N up to which the default
                                        engine takes it (the build parameter XENG_FUSED_MAX_N, 3584): no
                                        decode buffer, about 2% slower than two passes at N = 4096           */

typedef struct xeng_s *xeng_t;

/*
 * xeng_create -- make an X-engine for n_inputs inputs (N), n_freq channels
 * (F) and integrations of at most t_integ samples.
 *   Ranges: 1 <= N <= XENG_MAX_INPUTS, F >= 1, 1 <= t_integ <= XENG_MAX_T_INTEG
 *   (else XENG_ERR_RANGE).  Allocates the device accumulators
 *   (F * N(N+1)/2 * 8 bytes) and the tensor engine's decode buffer on the
 *   current CUDA device (XENG_ERR_NOMEM on failure).  *out_handle is set only
 *   on success.  Synchronous.
 */
XENG_API int xeng_create(int32_t n_inputs, int32_t n_freq, int64_t t_integ, xeng_t *out_handle);

/*
 * xeng_push -- integrate n_samples more samples (Sec. IV-C-1: integration).
 *   block: [n_samples][F][N] bytes, device memory or host memory (host memory
 *   is copied to the device on `stream` first; pinned host memory keeps the
 *   copy asynchronous).  The caller keeps `block` unchanged until `stream`
 *   has passed this call.  If samples already integrated + n_samples would
 *   exceed t_integ the call returns XENG_ERR_OVERFLOW and changes nothing.
 *   n_samples == 0 is a no-op.
 */
XENG_API int xeng_push(xeng_t h, const uint8_t *block, int64_t n_samples, void *stream);

/*
 * xeng_dump -- write the integrated triangle and start a new integration.
 *   out: [F][N(N+1)/2][2] int32, device or host memory.  With host memory
 *   the call returns after the data is in `out`; with device memory it is
 *   asynchronous on `stream`.  A dump with no samples integrated writes zeros.
 *   Returns the number of samples integrated (>= 0) or an XENG_ERR_* code.
 */
XENG_API int64_t xeng_dump(xeng_t h, int32_t *out, void *stream);

/*
 * xeng_correlate -- one whole integration in one call (Sec. IV-C-1): the
 *   visibilities of exactly these n_samples samples, written to `out`
 *   ([F][N(N+1)/2][2] int32), as xeng_push + xeng_dump on a fresh handle
 *   would give, but straight into `out` when it is device memory (no copy of
 *   the triangle; device `out` must be 8-byte aligned, else XENG_ERR_ARG).
 *   block as for xeng_push; n_samples <= t_integ (else XENG_ERR_OVERFLOW).  With device `out` the call is asynchronous on
 *   `stream` and leaves any integration in progress on the handle untouched;
 *   with host `out` it returns once the data is there, and needs the handle
 *   to have no integration in progress (else XENG_ERR_ARG).
 */
XENG_API int xeng_correlate(xeng_t h, const uint8_t *block, int64_t n_samples, int32_t *out, void *stream);

/*
 * xeng_correlate_gated -- one integration split into gates, with flagged
 *   samples excluded.  Gating (Sec. IV-C-4) partitions the samples by their
 *   time relative to a periodic source: gate[t] in [0, n_gates) names the
 *   sub-buffer of sample t (any other value drops it).  Flags (Sec. IV-A):
 *   valid[t][f][i] == 0 marks a missing or saturated sample, which then
 *   contributes nothing; the usable samples are counted per gate, channel and
 *   input for renormalising the integrated matrices downstream.
 *     V^g_ij(f) = sum over t with gate[t] == g, valid_i(t), valid_j(t) of x_i conj(x_j)
 *   block: device [n_samples][F][N]; gate: host int32 [n_samples];
 *   valid: device uint8 [n_samples][F][N] or NULL (all usable);
 *   out: device int32 [n_gates][F][N(N+1)/2][2] (overwritten, 8-byte aligned);
 *   counts: device int32 [n_gates][F][N] or NULL.
 *   n_samples <= min(t_integ, 65536) (else XENG_ERR_OVERFLOW / XENG_ERR_RANGE);
 *   tensor engine only.  Asynchronous on `stream` after reading `gate`.
 */
XENG_API int xeng_correlate_gated(xeng_t h, const uint8_t *block, int64_t n_samples, const int32_t *gate,
                                  int32_t n_gates, const uint8_t *valid, int32_t *out, int32_t *counts, void *stream);

/*
 * Gate accumulator sets (Sec. IV-C-4 gating, Sec. IV-A flagged data) kept on
 * the handle across pushes, so that one integration (e.g. 2^23 samples, Sec.
 * IV-C-1) is split into on/off sub-buffers by pulsar phase, each with the
 * number of usable samples per (gate, channel, input) for renormalising.
 *
 * xeng_set_gates -- give the handle n_gates accumulator sets (1 <=
 *   n_gates <= XENG_MAX_GATES, else XENG_ERR_RANGE) and their usable-sample
 *   counts, n_gates * F * N(N+1)/2 * 8 + n_gates * F * N * 4 bytes of device
 *   memory (XENG_ERR_NOMEM: the handle keeps one set).  Only with no
 *   integration in progress (else XENG_ERR_ARG).  Synchronizes the device.
 *   With one set (the default) xeng_push and xeng_dump work as always and
 *   plain pushes count every sample as usable; with more, xeng_push and
 *   xeng_dump return XENG_ERR_ARG and xeng_push_gated / xeng_dump_gated are
 *   the calls.
 *
 * xeng_push_gated -- integrate n_samples more samples of device block
 *   [n_samples][F][N] into the sets:
 *     V^g_ij(f) += sum over t with gate[t] == g, valid_i(t), valid_j(t) of x_i conj(x_j),
 *     counts[g][f][i] += #{t : gate[t] == g, valid_i(t)}.
 *   gate: host int32 [n_samples], a set per sample (values outside
 *   [0, n_gates) drop the sample), or NULL for set 0; valid: device uint8
 *   [n_samples][F][N] (0 = missing or saturated), or NULL for all usable.
 *   Any length (rounds of at most 65,536 samples per set); every sample
 *   counts against t_integ (XENG_ERR_OVERFLOW, nothing done).  Tensor engine
 *   only (else XENG_ERR_ARG), not while delays are set (XENG_ERR_UNSUPPORTED).
 *   Reads `gate` before returning and synchronizes `stream` (it uploads the
 *   per-set sample lists); the launches are asynchronous on `stream`.
 *
 * xeng_dump_gated -- write every set to out ([n_gates][F][N(N+1)/2][2]
 *   int32) and, if counts is not NULL, the usable-sample counts to counts
 *   ([n_gates][F][N] int32), device or host memory, then start a new
 *   integration.  Returns the samples pushed (>= 0) or an XENG_ERR_* code;
 *   returns once host buffers are written, else asynchronous on `stream`.
 */
#define XENG_MAX_GATES 64
XENG_API int xeng_set_gates(xeng_t h, int32_t n_gates);
XENG_API int xeng_push_gated(xeng_t h, const uint8_t *block, int64_t n_samples, const int32_t *gate,
                             const uint8_t *valid, void *stream);
XENG_API int64_t xeng_dump_gated(xeng_t h, int32_t *out, int32_t *counts, void *stream);

/*
 * xeng_set_delays -- time shifting (Sec. IV-C-5).  The signal of an outlying
 *   station reaches the correlator early relative to the other inputs, which
 *   decorrelates it from them; delaying that input by a whole number of
 *   samples restores the correlation.  With delays d_i set, every later
 *   xeng_push integrates
 *     V_ij(f) += sum_t y_i(t, f) conj(y_j(t, f)),   y_i(t, f) = x_i(t - d_i, f),
 *   where t counts the samples of the handle's stream (every push since this
 *   call, in order) and x_i(t) = 0 + 0i for t < 0.  Between pushes the handle
 *   keeps the last max(d) samples of each delayed input on the device
 *   (2 * max(d) * n_freq * #{i : d_i > 0} bytes); xeng_dump does not reset
 *   that history.
 *   delays: host int32 [n_inputs], each in [0, XENG_MAX_DELAY]; NULL, or all
 *   zero, removes the delays.  The history restarts empty (zeros) with every
 *   call.  Synchronizes the device: a set-up call, not for the streaming loop.
 *   Errors: XENG_ERR_ARG (NULL handle), XENG_ERR_RANGE (a delay out of range),
 *   XENG_ERR_UNSUPPORTED (handle on the dp4a engine), XENG_ERR_NOMEM (delays
 *   removed).  While delays are set, xeng_correlate, xeng_correlate_gated and
 *   xeng_set_engine(XENG_ENGINE_DP4A) return XENG_ERR_UNSUPPORTED: they have
 *   no stream history to shift against.
 */
#define XENG_MAX_DELAY 131072  /* samples; 168 ms at 2.56 us per sample is 65,625 */
XENG_API int xeng_set_delays(xeng_t h, const int32_t *delays);

/*
 * Beamforming (Sec. IV-C-3).  The telescope cannot point physically; a beam is
 * formed digitally by phase-shifting the inputs and summing them, so that
 * signals from a chosen sky direction add in phase, and is written out at the
 * full sample cadence.  For every sample t, channel f and beam b:
 *     y_b(t, f) = sum_i w_{f,b,i} x_i(t, f),   w = w_re + i w_im, int8 parts,
 * exact in int32 (|y| <= 2 * 128 * 8 * N < 2^31).
 *
 *   xbeam_create(n_inputs, n_freq, n_beams, &b): 16 <= n_inputs <= XENG_MAX_INPUTS
 *     with n_inputs a multiple of 16 (the block's rows are read by TMA, whose
 *     strides must be multiples of 16 bytes), 1 <= n_beams <= XBEAM_MAX_BEAMS;
 *     else XENG_ERR_RANGE.  All weights start at zero.
 *   xbeam_set_weights(b, w_re, w_im, stream): int8 [n_freq][n_beams][n_inputs]
 *     each, host or device memory (host: returns once they are copied).
 *   xbeam_run(b, block, n_samples, out, stream): block device uint8
 *     [n_samples][n_freq][n_inputs], 16-byte aligned; out device int32
 *     [n_samples][n_freq][n_beams][2] (Re, Im), 8-byte aligned, overwritten.
 *     Asynchronous on `stream`; a device-side time-out is reported by the next
 *     call as XENG_ERR_TIMEOUT (sticky).
 *   xbeam_destroy(b): synchronizes the device, frees the handle; NULL is a no-op.
 */
typedef struct xbeam_s *xbeam_t;
#define XBEAM_MAX_BEAMS 64
XENG_API int xbeam_create(int32_t n_inputs, int32_t n_freq, int32_t n_beams, xbeam_t *out);
XENG_API int xbeam_set_weights(xbeam_t b, const int8_t *w_re, const int8_t *w_im, void *stream);
XENG_API int xbeam_run(xbeam_t b, const uint8_t *block, int64_t n_samples, int32_t *out, void *stream);
XENG_API void xbeam_destroy(xbeam_t b);

/* xeng_destroy -- free the handle and its device memory; NULL is a no-op.
 * Synchronizes the device first. */
XENG_API void xeng_destroy(xeng_t h);

/* xeng_strerror -- static text for a status code. */
XENG_API const char *xeng_strerror(int code);

/*
 * xeng_set_engine -- choose XENG_ENGINE_TENSOR, XENG_ENGINE_DP4A,
 *   XENG_ENGINE_TENSOR_PLANES or XENG_ENGINE_TENSOR_FUSED for the following
 *   pushes (XENG_ERR_ARG for other values).  All engines add into the same
 *   int32 accumulators, so an integration may mix them.
 */
XENG_API int xeng_set_engine(xeng_t h, int32_t engine);

/*
 * xeng_decode -- the standalone nibble-unpack / offset-decode stage (Sec.
 *   II-A footnote) as the tensor engine runs it: channels [f0, f0 + nf) and
 *   samples [0, n_samples) of block [n_samples][F][N] (device memory) become
 *   FP8 E4M3 codes of the integer values in
 *     planes [nf][2][n_pad][t_pad]   (plane 0 = real parts, 1 = imaginary)
 *   with n_pad = N rounded up to 128 and t_pad = n_samples rounded up to 128;
 *   padding is written as code 0x00 (+0.0).  planes is device memory of
 *   nf * 2 * n_pad * t_pad bytes.  Where N is a multiple of 16 and block is
 *   16-byte aligned the stage runs as the engine's TMA pipeline and the call
 *   synchronizes `stream`, returning XENG_ERR_TIMEOUT if the pipeline stalled
 *   (bounded waits, 2 s); otherwise it is asynchronous on `stream`.
 */
XENG_API int xeng_decode(const uint8_t *block, int64_t n_samples, int32_t n_freq, int32_t n_inputs,
                         int32_t f0, int32_t nf, uint8_t *planes, void *stream);

/*
 * xeng_selftest_wait_timeout -- exercise the kernels' bounded waits without a
 *   fault or a hang: one thread of a 64-thread kernel waits limit_ns
 *   (<= 1 s) on a barrier nothing completes, gives up and writes the
 *   time-out status (2) to the status word; the other 63 threads, waiting on
 *   the same barrier with the kernels' 2 s limit, see the word and leave at
 *   once.  Writes the final status word and the number of threads that gave
 *   up (64).  Synchronous; allocates 8 bytes.
 */
XENG_API int xeng_selftest_wait_timeout(int64_t limit_ns, int32_t *status, int32_t *threads_left);

/* Launch and device-time counters of one handle (see xeng_set_profiling). */
typedef struct {
    int64_t launches;          /* kernels launched by this handle so far      */
    int64_t decode_launches;   /* ... of which decode kernels                 */
    int64_t correlate_launches;/* ... of which correlation kernels            */
    double  decode_ms;         /* summed device time of timed decode launches */
    double  correlate_ms;      /* summed device time of timed correlations    */
    int64_t timed_decode;      /* decode launches included in decode_ms       */
    int64_t timed_correlate;   /* correlation launches in correlate_ms        */
} xeng_stats_t;

/*
 * xeng_set_profiling -- on != 0: bracket every kernel this handle launches
 *   with CUDA events on its stream, so xeng_get_stats can report device
 *   times per kernel kind.  Off by default.
 */
XENG_API int xeng_set_profiling(xeng_t h, int32_t on);

/*
 * xeng_get_stats -- copy the counters into *stats.  If reset != 0, zero them
 *   afterwards.  Waits for the timed launches to finish.
 */
XENG_API int xeng_get_stats(xeng_t h, xeng_stats_t *stats, int32_t reset);

/*
 * Batches: many independent whole integrations (Sec. IV-C-1) of uneven
 * sizes -- different N, F and T per job -- planned once and then run as one
 * persistent decode launch (a second one only for jobs with N not a multiple
 * of 16 or an unaligned block) plus one persistent tensor-core launch,
 * captured in a CUDA graph.  Every job's result is bit-identical to correlating it alone.
 */
typedef struct {
    int32_t n_inputs;       /* N of this job, 1..XENG_MAX_INPUTS                  */
    int32_t n_freq;         /* F of this job, >= 1                                */
    int64_t n_samples;      /* T of this job, 1..XENG_MAX_T_INTEG                 */
    const uint8_t *block;   /* device memory [T][F][N], caller-owned              */
    int32_t *out;           /* device memory [F][N(N+1)/2][2] int32, caller-owned, 8-byte aligned */
} xeng_job_t;

#define XENG_SCHED_LPT         0  /* longest items first onto the least-loaded CTA */
#define XENG_SCHED_ROUND_ROBIN 1  /* items dealt round-robin in job order          */
#define XENG_SCHED_ORDERED     2  /* items in job order, each to the CTA expected to be
                                     free first: CTAs stay on neighbouring tiles       */

#define XENG_TILES_ROW_MAJOR 0  /* a channel's tile pairs (I <= J) row by row              */
#define XENG_TILES_DIAGONAL  1  /* by diagonal J - I, the main diagonal first              */
#define XENG_TILES_MORTON    2  /* in Z order of (I, J): neighbouring tiles share operands */

typedef struct {
    int32_t max_chunks_per_item; /* split a tile's integration into items of at most this many
                                    128-sample chunks (1..512; <= 0 means 512)            */
    int32_t policy;              /* XENG_SCHED_LPT, _ROUND_ROBIN or _ORDERED               */
    int32_t use_graph;           /* != 0: capture the run in a CUDA graph once, replay it */
    int32_t tile_order;          /* XENG_TILES_ROW_MAJOR, _DIAGONAL or _MORTON            */
} xeng_batch_opts_t;

typedef struct {
    int32_t n_jobs;
    int64_t n_items;             /* work items of the persistent launch                  */
    int32_t grid;                /* persistent CTAs (one per SM)                         */
    int64_t decode_ctas;         /* 128 x 128 tiles the decode launches convert per run  */
    int64_t planes_bytes;        /* decode scratch owned by the batch                    */
    int32_t max_chunks_per_item;
    int32_t policy;
    double  load_imbalance;      /* planned max / mean CTA load                          */
    int32_t tile_order;
} xeng_batch_info_t;

typedef struct xeng_batch_s *xeng_batch_t;

/*
 * xeng_batch_create -- plan a batch over jobs[0..n_jobs) on the current
 *   device: allocates the decode scratch (about twice the jobs' input bytes),
 *   per-job TMA descriptors and the work list, and (use_graph) captures the
 *   run in a CUDA graph.  The block and out pointers are bound now and used by
 *   every run.  opts may be NULL (LPT, 512 chunks, graph, row-major tiles).
 *   Synchronous.  XENG_ERR_ARG for NULL or host pointers or an unknown policy
 *   or tile order, XENG_ERR_RANGE for bad sizes.
 */
XENG_API int xeng_batch_create(const xeng_job_t *jobs, int32_t n_jobs, const xeng_batch_opts_t *opts,
                               xeng_batch_t *out_batch);

/* xeng_batch_run -- enqueue one run on `stream`: every job's visibilities of
 *   its whole block are written to its out (overwritten).  Asynchronous; a
 *   device-side time-out of an earlier run is reported as XENG_ERR_TIMEOUT. */
XENG_API int xeng_batch_run(xeng_batch_t b, void *stream);

/* xeng_batch_info -- the plan's sizes and its predicted load balance. */
XENG_API int xeng_batch_info(xeng_batch_t b, xeng_batch_info_t *info);

/* xeng_batch_destroy -- free the batch (synchronizes the device); NULL is a no-op. */
XENG_API void xeng_batch_destroy(xeng_batch_t b);

/*
 * xeng_batch_autotune -- pick xeng_batch_opts_t for these jobs by timing every
 *   (max_chunks_per_item in {16, 32, 64, 128, 256, 512}) x (policy) candidate
 *   with row-major tiles for `reps` runs each, in two passes (forward, then
 *   reverse order; each candidate keeps its better time), then the winner with
 *   the diagonal and Morton tile orders, overwriting the jobs' outputs.  With
 *   a cache_path, a JSON-lines file of {"sig", "max_chunks", "policy",
 *   "tile_order", "ms"} records keyed by the jobs' (N, F, T) list and the SM
 *   count is read first (hit: returns 1 without timing) and the winner
 *   appended after tuning (returns 0).  *best_ms (may be NULL) receives the
 *   winner's time per run.  Negative XENG_ERR_* on error.
 */
XENG_API int xeng_batch_autotune(const xeng_job_t *jobs, int32_t n_jobs, const char *cache_path, int32_t reps,
                                 xeng_batch_opts_t *best, double *best_ms);

/*
 * Streaming service: frame blocks from many concurrent streams, integrated
 * continuously into device-resident accumulators (Sec. IV-A data flow,
 * Sec. IV-C-1 integration) and dumped on a fixed cadence.  A worker thread
 * batches whatever blocks are queued across all streams into each round (one
 * decode launch + one persistent tensor-core launch), with up to two rounds in
 * flight; blocks that arrive meanwhile join the next round.  Streams are
 * admitted against an HBM budget (accumulators, two dump buffers and two
 * decode slices each) and, optionally, a compute budget; closing a stream
 * frees its share for later admissions.  Results are bit-identical to
 * integrating each stream alone.
 *
 * Lost and late blocks (Sec. IV-A: momentary faults must not stop the data
 * gathering).  Block number b of a stream (0, 1, 2, ... in the order the
 * stream produced them) belongs to integration b / (dump_samples /
 * block_samples).  An integration closes when all of its blocks are
 * integrated, when a block of a later integration reaches the head of the
 * stream's queue, or after xserve_flush; it is then dumped with the blocks it
 * has (xserve_dump_info_t.blocks, .missing_blocks; integrations that received
 * no block at all produce no dump).  A block of an integration that a later
 * block has already closed is refused with XENG_ERR_LATE and counted.
 */
typedef struct xserve_s *xserve_t;

typedef struct {
    int64_t hbm_budget_bytes;    /* device memory streams may hold (default 120 GiB)             */
    int32_t max_blocks;          /* blocks of one stream per round (default 16)                  */
    int32_t max_streams;         /* stream slots (default 16)                                    */
    int64_t max_items;           /* tile pairs one round may hold (default 4 Mi)                  */
    double  compute_budget_tops; /* > 0: also refuse streams whose declared demand exceeds it     */
} xserve_opts_t;

typedef struct {
    int64_t seq;                 /* integration number of the stream (0, 1, ...)                  */
    int64_t samples;             /* samples integrated (dump_samples unless blocks were lost)     */
    double  last_arrival_s;      /* arrival time of the integration's last block (xserve_now clock) */
    double  ready_s;             /* time the dump was seen complete                               */
    int64_t blocks;              /* blocks integrated                                             */
    int64_t missing_blocks;      /* blocks of the integration never integrated (lost or late)     */
} xserve_dump_info_t;

typedef struct {
    int64_t rounds, blocks_done, dumps_done, refused, backlog_blocks, used_bytes;
    int32_t open_streams, pad_;
    double  useful_ops;          /* 8 ops per complex MAC over all integrated blocks             */
    double  busy_s;              /* first arrival -> last completed round                         */
    double  block_p50_s, block_p99_s;  /* block arrival -> its round complete                     */
    double  dump_p50_s, dump_p99_s;    /* last block of an integration -> dump available          */
    double  gpu_decode_ms, gpu_correlate_ms;  /* summed device time of the rounds' decode and of
                                                 their correlation (the single-pass launches too) */
    double  host_plan_ms;                     /* summed host time spent building rounds           */
    int64_t late_blocks;                      /* blocks refused with XENG_ERR_LATE                */
    int64_t short_dumps;                      /* dumps of integrations closed with blocks missing */
} xserve_stats_t;

/* xserve_now -- the server's clock (seconds, monotonic) for arrival stamps. */
XENG_API double xserve_now(void);

/* xserve_create -- start a server and its worker thread on the current device;
 *   opts may be NULL for the defaults. */
XENG_API int xserve_create(const xserve_opts_t *opts, xserve_t *out);

/*
 * xserve_open_stream -- admit a stream of n_inputs x n_freq blocks of
 *   block_samples samples, dumped every dump_samples samples (a multiple of
 *   block_samples, <= XENG_MAX_T_INTEG; block_samples rounded up to 128 times
 *   max_blocks must be <= 65536).  rate_blocks_per_s is the declared arrival
 *   rate, used only by the compute budget.  Returns XENG_ERR_NOMEM when the
 *   budget (or a slot) is not available now -- retry after another stream
 *   closes -- and sets *stream_id on success.  A stream whose rounds the
 *   single-pass kernels take (N a multiple of 16 up to 3584, block_samples a
 *   multiple of 128 and <= 32768; unless the environment variable
 *   XENG_FUSED_KERNEL was "none" when the server was created) reads its blocks
 *   in place: it holds no decode planes (its HBM charge is its accumulators and
 *   two dump buffers) and its blocks must be 16-byte aligned.
 */
XENG_API int xserve_open_stream(xserve_t sv, int32_t n_inputs, int32_t n_freq, int64_t block_samples,
                                int64_t dump_samples, double rate_blocks_per_s, int32_t *stream_id);

/*
 * xserve_submit -- queue one block ([block_samples][F][N] bytes, device
 *   memory) that arrived at arrival_s (xserve_now clock; <= 0 = now), as the
 *   block after the highest-numbered one submitted so far.  Never waits for
 *   the GPU.  The caller keeps the block unchanged until xserve_consumed
 *   reports it (blocks of a stream are consumed in queue order).  XENG_ERR_ARG
 *   for a block of a single-pass stream (see xserve_open_stream) that is not
 *   16-byte aligned.
 */
XENG_API int xserve_submit(xserve_t sv, int32_t stream_id, const uint8_t *block, double arrival_s);

/*
 * xserve_submit_seq -- as xserve_submit, for block number seq (>= 0) of the
 *   stream, so that lost blocks leave gaps.  Returns XENG_ERR_LATE (block not
 *   queued) if a block of a later integration was submitted before it, and
 *   XENG_ERR_ARG if block number seq was already submitted.
 */
XENG_API int xserve_submit_seq(xserve_t sv, int32_t stream_id, const uint8_t *block, int64_t seq, double arrival_s);

/*
 * xserve_flush -- close the stream's newest integration once the blocks
 *   queued before this call are integrated, even if blocks are missing (for
 *   example at the end of an observation); later blocks start the next one.
 */
XENG_API int xserve_flush(xserve_t sv, int32_t stream_id);

/* xserve_consumed -- blocks of the stream whose round has completed. */
XENG_API int64_t xserve_consumed(xserve_t sv, int32_t stream_id);

/*
 * xserve_poll_dump -- if the stream's oldest finished integration is ready,
 *   copy its [F][N(N+1)/2][2] int32 triangle to out (host or device memory),
 *   fill *info (may be NULL) and return 1; else return 0.  A stream whose two
 *   dump buffers are both full waits for its dumps to be taken.
 */
XENG_API int xserve_poll_dump(xserve_t sv, int32_t stream_id, int32_t *out, xserve_dump_info_t *info);

/* xserve_drain -- wait (up to timeout_s; <= 0 = no limit) until every queued
 *   block that can run has been integrated. */
XENG_API int xserve_drain(xserve_t sv, double timeout_s);

/* xserve_close_stream -- drop its queued blocks, wait for its rounds in
 *   flight, free its device memory and budget. */
XENG_API int xserve_close_stream(xserve_t sv, int32_t stream_id);

/* xserve_stats -- counters and latency percentiles so far. */
XENG_API int xserve_stats(xserve_t sv, xserve_stats_t *out);

/* xserve_destroy -- stop the worker (queued blocks are dropped) and free everything. */
XENG_API void xserve_destroy(xserve_t sv);

/* Size of the decode area of the fixed device array xeng_correlate_noalloc
 * works in (64 MiB; the array holds 256 bytes more for a status word). */
#define XENG_NOALLOC_SCRATCH_BYTES 67108864LL

/*
 * xeng_correlate_noalloc -- one whole integration of `block` into `out`,
 *   computed like xeng_push + xeng_dump on a fresh handle with the tensor
 *   engine, but without allocating any device memory.  The paper has no
 *   counterpart: this is for callers that cannot allocate at the point where
 *   they correlate -- e.g. a real-time capture loop whose device memory was
 *   divided up once at start-up by its own pool, or a loop that cannot afford
 *   the device-wide synchronization cudaMalloc / cudaFree may cause.
 *
 *   block: [n_samples][n_freq][n_inputs] bytes, device memory (caller-owned).
 *   out:   [n_freq][N(N+1)/2][2] int32, device memory (caller-owned),
 *          8-byte aligned; overwritten (n_samples == 0 writes zeros).
 *   Working memory is one library-owned __device__ array of
 *   XENG_NOALLOC_SCRATCH_BYTES + 256 bytes that each GPU loading the library
 *   holds until the process exits.  Sizes beyond what it holds are rejected
 *   with XENG_ERR_RANGE: n_samples <= 65536 and
 *   2 * round_up(N, 128) * round_up(n_samples, 128) <= XENG_NOALLOC_SCRATCH_BYTES
 *   (e.g. N = 2048 with 16384 samples, or N = 256 with 65536 samples).
 *   Host pointers give XENG_ERR_ARG.  The call enqueues its work on `stream`
 *   and returns once it is done (it synchronizes `stream`); a device-side
 *   wait time-out gives XENG_ERR_TIMEOUT.  It calls no cudaMalloc, cudaFree
 *   or other allocating routine.
 *   The first call on a device looks up the array's device address with that
 *   device current; make that first call before any stream capture.  That
 *   address is kept for the life of the process and does not survive
 *   cudaDeviceReset: do not call this entry point on a device after
 *   resetting it.  All
 *   calls on a device share the array: calls that overlap on the GPU (from
 *   several threads or streams) race and give wrong results.
 */
XENG_API int xeng_correlate_noalloc(const uint8_t *block, int64_t n_samples, int32_t n_freq, int32_t n_inputs,
                                    int32_t *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* XENG_H */
