// single_pass.cu -- which of the single-pass kernels (the nibble split of paper
// Sec. II-A fused into the correlation of Sec. IV-C-1) takes a block of N
// inputs, and their common launch, for handles and batches alike.
#include <cstdlib>
#include <cstring>

#include "xeng_internal.h"

namespace xeng {

// Up to 256 inputs: single CTAs over the upper-triangle 128-input blocks
// (correlate_small.cu).  0 disables it (such blocks decode to planes).
#ifndef XENG_FUSED_SMALL
#define XENG_FUSED_SMALL 1
#endif
// Above 256 inputs the single pass runs either the 2-CTA pair kernel over
// 256-input block pairs (correlate_pair.cu) or single CTAs over 128-input block
// pairs (correlate_onepass.cu), whichever costs less by the measured time of
// one block pair (GB300, 1024 channels x 8192 samples: 1.09-1.20 ms per 256 x
// 256 pair, 0.35-0.44 ms per 128 x 128 pair, in units of 10 us).  The pair
// kernel does a quarter of the MMAs per block in a quarter of the items, but
// pads N to 256: it wins unless ceil(N / 128) is odd, and the one pass's cost
// per pair grows above about 1900 inputs (one pass / pair, ms: N = 384 2.35 /
// 3.22; 512 3.66 / 3.26; 640 5.26 / 6.75; 768 7.50 / 6.75; 896 9.79 / 11.05;
// 1024 13.06 / 11.09; 1152 15.98 / 16.96; 1408 23.15 / 23.90; 1664 32.13 /
// 33.70; 1920 51.88 / 42.12; 2176 67.87 / 53.46: the ratio of the two costs
// must lie between 3.25 and 3.33).  A cost of 0 forces that kernel.
#ifndef XENG_PAIR_COST
#define XENG_PAIR_COST 118
#endif
#ifndef XENG_ONEPASS_COST
#define XENG_ONEPASS_COST 36
#endif
// Above this many inputs the default engine and batches decode to planes first
// (two passes) instead of the single pass: the decode pass grows with N, the
// correlation with N^2, and the plane GEMM does a block pair about 15% faster
// than the pair kernel's converters feed it (GB300, 8192 samples, ms single /
// two passes: N = 2048 x 1024 channels 43.5 / 45.1, N = 3072 x 512 46.8 / 47.7,
// N = 4096 x 256 40.8 / 40.0; a fit of both puts the crossover near 3600).
#ifndef XENG_FUSED_MAX_N
#define XENG_FUSED_MAX_N 3584
#endif

namespace {

bool use_pair_kernel(int32_t N)
{
    const int64_t b2 = (N + 255) / 256, b1 = (N + 127) / 128;
    return (int64_t)XENG_PAIR_COST * (b2 * (b2 + 1) / 2) < (int64_t)XENG_ONEPASS_COST * (b1 * (b1 + 1) / 2);
}

}  // namespace

int single_pass_force_from_env()
{
    const char *env = getenv("XENG_FUSED_KERNEL");
    if (!env) return 0;
    if (!strcmp(env, "pair")) return kSinglePair;
    if (!strcmp(env, "onepass")) return kSingleOnepass;
    if (!strcmp(env, "none")) return kSingleNone;
    return 0;
}

int single_pass_kernel(const uint8_t *block, int32_t N, int force, bool bounded)
{
    if (force == kSingleNone || (bounded && N > XENG_FUSED_MAX_N)) return 0;
    const int k = force ? force : N <= 256 ? kSingleSmall : use_pair_kernel(N) ? kSinglePair : kSingleOnepass;
    switch (k) {
    case kSingleSmall: return XENG_FUSED_SMALL && small_ok(block, N) ? k : 0;
    case kSinglePair: return pair_ok(block, N) ? k : 0;
    default: return onepass_ok(block, N) ? k : 0;
    }
}

cudaError_t small_scratch_alloc(SmallScratch *sc, int num_sms, cudaStream_t s)
{
    if (sc->ws) return cudaSuccess;
    cudaError_t e = cudaMalloc(&sc->ws, small_ws_bytes(num_sms));
    if (e == cudaSuccess) e = cudaMalloc(&sc->flags, small_flags_bytes(num_sms));
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->flags, 0, small_flags_bytes(num_sms), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        small_scratch_free(sc);
    }
    return e;
}

void small_scratch_free(SmallScratch *sc)
{
    cudaFree(sc->ws);
    cudaFree(sc->flags);
    sc->ws = nullptr;
    sc->flags = nullptr;
}

cudaError_t launch_single_pass(int kernel, const uint8_t *block, int64_t T_block, int64_t t0, int64_t nt, int32_t F,
                               int32_t N, int32_t f0, int32_t nf, int32_t *acc, int accumulate, SmallScratch *sc,
                               int *err, int num_sms, cudaStream_t s, const CUtensorMap *maps, int32_t spb)
{
    if (kernel == kSingleSmall) {
        cudaError_t e = small_scratch_alloc(sc, num_sms, s);
        if (e != cudaSuccess) return e;
        return launch_correlate_small(block, T_block, t0, nt, F, N, f0, nf, acc, accumulate, sc->ws, sc->flags, err,
                                      num_sms, s, maps, spb);
    }
    if (kernel == kSinglePair)
        return launch_correlate_pair(block, T_block, t0, nt, F, N, f0, nf, acc, accumulate, err, num_sms, s, maps,
                                     spb);
    if (kernel == kSingleOnepass)
        return launch_correlate_onepass(block, T_block, t0, nt, F, N, f0, nf, acc, accumulate, err, num_sms, s, maps,
                                        spb);
    return cudaErrorInvalidValue;
}

cudaError_t encode_single_pass_map(int kernel, CUtensorMap *map, const uint8_t *block, int64_t T_block, int32_t F,
                                   int32_t N)
{
    if (kernel == kSingleSmall) return encode_small_map(map, block, T_block, F, N);
    if (kernel == kSinglePair) return encode_pair_map(map, block, T_block, F, N);
    if (kernel == kSingleOnepass) return encode_onepass_map(map, block, T_block, F, N);
    return cudaErrorInvalidValue;
}

int single_pass_stage(int kernel)
{
    if (kernel == kSingleSmall) return small_stage_samples();
    if (kernel == kSinglePair) return pair_stage_samples();
    if (kernel == kSingleOnepass) return onepass_stage_samples();
    return 0;
}

}  // namespace xeng
