// xeng_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace xeng {

constexpr int kTile = 128;          // inputs per tensor-engine tile, samples per K chunk
constexpr int kMaxChunkSamples = 65536;  // f32 sums stay <= 128 * 65536 = 2^23 (exact)

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
};
cudaError_t launch_correlate_tc(const TcArgs &a, int num_sms, cudaStream_t s);

// Plain CUDA-core correlation straight from the bytes (dp4a, int32).
cudaError_t launch_correlate_dp4a(const uint8_t *block, int64_t T, int32_t F, int32_t N,
                                  int32_t *acc, int32_t accumulate, cudaStream_t s);

}  // namespace xeng
