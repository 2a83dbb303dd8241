// decode.cu -- nibble unpack and offset decode (paper Sec. II-A and its
// footnote: each 4-bit nibble stores value + 8, values in [-8, 7]; high
// nibble = real part, low nibble = imaginary part), producing the tensor
// engine's operands.
//
// In:  block  [T][F][N] bytes (input index fastest).
// Out: planes [nf][2][n_pad][t_pad] bytes: for channel f0 + fl, plane 0 holds
//      the real parts and plane 1 the imaginary parts, one row per input,
//      samples contiguous ("K-major" for the correlation GEMM), each value
//      as its FP8 E4M3 code.  Integers -8..7 are exact in E4M3.  Rows i >= N
//      and samples t >= T are written as +0.0.
//
// One CTA transposes and decodes a 128-sample x 128-input tile of one
// channel: coalesced 16-byte loads into shared memory, then each thread
// takes 4 inputs x 16 samples, transposes 4x4 byte blocks with byte permutes,
// decodes through half precision (the nibble is placed in the mantissa of
// 1024.0, so the half value is 1024 + u, minus 1032 gives u - 8 exactly) and
// packs pairs to E4M3 with the hardware converter.  HBM-bound: 1 byte read,
// 2 bytes written per (input, sample).
#include "nibble.cuh"
#include "xeng_internal.h"

namespace xeng {
namespace {

constexpr int kDecThreads = 256;
constexpr int kRowWords = 33;  // 128 bytes + 4 bytes of padding per sample row
// Row t of the shared tile starts at word t * 33 + (t / 16) * 4: the extra
// skew per 16-row group keeps the column reads of phase 2 conflict-free.
__device__ __forceinline__ int row_word(int t) { return t * kRowWords + (t >> 4) * 4; }
constexpr int kTileWords = 128 * kRowWords + 8 * 4;

// Phase 2 of a tile (after the 128 x 128 bytes sit in `tile`): thread =
// (input quad q, 16-sample block b); transpose, decode, store both planes.
__device__ __forceinline__ void decode_tile_store(const uint32_t *tile, uint8_t *__restrict__ planes, int64_t pitch,
                                                  int64_t n_pad, int64_t t0, int i0, int fl)
{
    const int tid = threadIdx.x;
    const int b = tid & 7;    // lanes 0..7 of a row group write one 128-byte row segment
    const int q = tid >> 3;   // 0..31
    uint32_t re[4][4], im[4][4];  // [input k][word g] (word g = samples 4g..4g+3)
    #pragma unroll
    for (int g = 0; g < 4; g++) {
        uint32_t r[4];
        #pragma unroll
        for (int k = 0; k < 4; k++) r[k] = tile[row_word(b * 16 + g * 4 + k) + q];
        // transpose + decode: r[k] byte m = (sample k, input m) -> input m's codes of samples 0..3
        decode_input4(r, 0, re[0][g], im[0][g]);
        decode_input4(r, 1, re[1][g], im[1][g]);
        decode_input4(r, 2, re[2][g], im[2][g]);
        decode_input4(r, 3, re[3][g], im[3][g]);
    }
    const int64_t tcol = t0 + b * 16;
    #pragma unroll
    for (int k = 0; k < 4; k++) {
        const int64_t i = i0 + q * 4 + k;
        uint8_t *rowre = planes + ((int64_t)fl * 2 * n_pad + i) * pitch + tcol;
        uint8_t *rowim = planes + ((int64_t)fl * 2 * n_pad + n_pad + i) * pitch + tcol;
        *reinterpret_cast<uint4 *>(rowre) = make_uint4(re[k][0], re[k][1], re[k][2], re[k][3]);
        *reinterpret_cast<uint4 *>(rowim) = make_uint4(im[k][0], im[k][1], im[k][2], im[k][3]);
    }
}

// Decode one 128-sample x 128-input tile (tb, ib) of channel f0 + fl into
// planes whose rows are `pitch` bytes apart.
__device__ __forceinline__ void decode_tile(const uint8_t *__restrict__ block, int64_t T, int32_t F, int32_t N,
                                            int32_t f0, uint8_t *__restrict__ planes, int64_t pitch, int64_t n_pad,
                                            int vec_ok, int tb, int ib, int fl, uint32_t *tile)
{
    const int64_t t0 = (int64_t)tb * 128;
    const int i0 = ib * 128;
    const int64_t f = f0 + fl;
    const int tid = threadIdx.x;

    // Phase 1: 128 rows x 8 chunks of 16 bytes; value 0x88 (0 + 0i) outside.
    for (int ch = tid; ch < 128 * 8; ch += kDecThreads) {
        const int t = ch >> 3, c = ch & 7;
        const int64_t tt = t0 + t;
        const int ic = i0 + c * 16;
        uint32_t w[4];
        if (tt < T && vec_ok && ic + 16 <= N) {
            const uint4 v = *reinterpret_cast<const uint4 *>(block + (tt * F + f) * N + ic);
            w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
        } else {
            for (int k = 0; k < 4; k++) {
                uint32_t word = 0;
                for (int b = 0; b < 4; b++) {
                    const int i = ic + k * 4 + b;
                    uint32_t byte = 0x88;
                    if (tt < T && i < N) byte = block[(tt * F + f) * N + i];
                    word |= byte << (8 * b);
                }
                w[k] = word;
            }
        }
        uint32_t *dst = tile + row_word(t) + c * 4;
        dst[0] = w[0]; dst[1] = w[1]; dst[2] = w[2]; dst[3] = w[3];
    }
    __syncthreads();

    decode_tile_store(tile, planes, pitch, n_pad, t0, i0, fl);
}

__global__ void __launch_bounds__(kDecThreads)
decode_kernel(const uint8_t *__restrict__ block, int64_t T, int32_t F, int32_t N, int32_t f0,
              uint8_t *__restrict__ planes, int64_t t_pad, int64_t n_pad, int vec_ok)
{
    __shared__ uint32_t tile[kTileWords];
    decode_tile(block, T, F, N, f0, planes, t_pad, n_pad, vec_ok, blockIdx.x, blockIdx.y, blockIdx.z, tile);
}

// All jobs of a batch in one launch: CTA b belongs to the job j with
// cta0[j] <= b < cta0[j + 1] and takes that job's tile b - cta0[j].
__global__ void __launch_bounds__(kDecThreads)
decode_batch_kernel(const DecodeJob *__restrict__ jobs, int n_jobs)
{
    __shared__ uint32_t tile[kTileWords];
    const int64_t b = blockIdx.x;
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {  // last job whose first CTA is <= b
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].cta0 <= b) lo = mid;
        else hi = mid - 1;
    }
    const DecodeJob &j = jobs[lo];
    const int64_t local = b - j.cta0;
    const int64_t ntb = j.t_pad / 128, nib = j.n_pad / 128;
    const int tb = (int)(local % ntb);
    const int ib = (int)((local / ntb) % nib);
    const int fl = (int)(local / (ntb * nib));
    decode_tile(j.block, j.T, j.F, j.N, 0, j.planes, j.pitch, j.n_pad, j.vec_ok, tb, ib, fl, tile);
}


// Gated, flagged decode: the tile's samples are rows idx[t0 .. t0 + 127] of the
// block (the samples of one gate, in order); a sample whose valid byte is 0 is
// replaced by value 0 + 0i, and the usable samples per input are added to
// counts[fl * N + i].  Rows past Tg and inputs past N decode to +0.0.
__global__ void __launch_bounds__(kDecThreads)
decode_gather_kernel(const uint8_t *__restrict__ block, int32_t F, int32_t N, int32_t f0,
                     const int32_t *__restrict__ idx, int64_t Tg, const uint8_t *__restrict__ valid,
                     uint8_t *__restrict__ planes, int64_t t_pad, int64_t n_pad, int32_t *__restrict__ counts,
                     int vec_ok)
{
    __shared__ uint32_t tile[kTileWords];
    __shared__ int cnt[128];
    const int64_t t0 = (int64_t)blockIdx.x * 128;
    const int i0 = blockIdx.y * 128;
    const int fl = blockIdx.z;
    const int64_t f = f0 + fl;
    const int tid = threadIdx.x;
    if (tid < 128) cnt[tid] = 0;
    __syncthreads();
    // usable-sample counters of this thread's 16 inputs (its chunk c = tid & 7
    // is the same for all its rows), one byte each, four to a word
    uint32_t acc[4] = {0u, 0u, 0u, 0u};
    for (int ch = tid; ch < 128 * 8; ch += kDecThreads) {
        const int t = ch >> 3, c = ch & 7;
        const int64_t k = t0 + t;
        const int ic = i0 + c * 16;
        uint32_t w[4] = {0x88888888u, 0x88888888u, 0x88888888u, 0x88888888u};
        if (k < Tg) {
            const int64_t row = ((int64_t)idx[k] * F + f) * N;
            if (vec_ok && ic + 16 <= N) {
                // 16 bytes of samples and 16 validity bytes at once; a flagged
                // byte becomes 0x88 (value 0 + 0i)
                const uint4 x = *reinterpret_cast<const uint4 *>(block + row + ic);
                w[0] = x.x; w[1] = x.y; w[2] = x.z; w[3] = x.w;
                if (valid) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(valid + row + ic);
                    const uint32_t vw[4] = {v.x, v.y, v.z, v.w};
                    #pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const uint32_t z = __vcmpeq4(vw[j], 0u);  // 0xFF in each flagged byte
                        w[j] = (w[j] & ~z) | (0x88888888u & z);
                        acc[j] += ~z & 0x01010101u;
                    }
                } else {
                    #pragma unroll
                    for (int j = 0; j < 4; j++) acc[j] += 0x01010101u;
                }
            } else {
                for (int m = 0; m < 16; m++) {
                    const int i = ic + m;
                    if (i >= N) break;
                    uint32_t byte = block[row + i];
                    if (valid && !valid[row + i]) byte = 0x88;
                    else acc[m >> 2] += 1u << (8 * (m & 3));
                    w[m >> 2] = (w[m >> 2] & ~(0xFFu << (8 * (m & 3)))) | (byte << (8 * (m & 3)));
                }
            }
        }
        uint32_t *dst = tile + row_word(t) + c * 4;
        dst[0] = w[0]; dst[1] = w[1]; dst[2] = w[2]; dst[3] = w[3];
    }
    if (counts) {
        // lanes l, l ^ 8, l ^ 16, l ^ 24 hold the same chunk: sum them (each byte
        // counter stays <= 16), then one lane per chunk adds into shared memory
        const int lane = tid & 31;
        #pragma unroll
        for (int j = 0; j < 4; j++) {
            acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], 8);
            acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], 16);
        }
        if (lane < 8) {
            #pragma unroll
            for (int m = 0; m < 16; m++) {
                const int n = (int)((acc[m >> 2] >> (8 * (m & 3))) & 0xFFu);
                if (n) atomicAdd(&cnt[(tid & 7) * 16 + m], n);
            }
        }
    }
    __syncthreads();
    decode_tile_store(tile, planes, t_pad, n_pad, t0, i0, fl);
    if (counts && tid < 128 && i0 + tid < N && cnt[tid]) atomicAdd(&counts[(int64_t)fl * N + i0 + tid], cnt[tid]);
}

// Shifted decode (Sec. IV-C-5): plane column t of input i holds the sample
// t0 + t - d_i of the block, or of the history when that index is negative.
// A 16-input chunk whose inputs share one delay keeps the 16-byte load.
__global__ void __launch_bounds__(kDecThreads)
decode_shifted_kernel(const uint8_t *__restrict__ block, int64_t t0, int64_t nt, int32_t F, int32_t N, int32_t f0,
                      const ShiftArgs sa, uint8_t *__restrict__ planes, int64_t t_pad, int64_t n_pad, int vec_ok)
{
    __shared__ uint32_t tile[kTileWords];
    const int64_t tr0 = (int64_t)blockIdx.x * 128;  // first plane column of the tile
    const int i0 = blockIdx.y * 128;
    const int fl = blockIdx.z;
    const int64_t f = f0 + fl;
    const int tid = threadIdx.x;
    for (int ch = tid; ch < 128 * 8; ch += kDecThreads) {
        const int t = ch >> 3, c = ch & 7;
        const int64_t tt = t0 + tr0 + t;  // sample of the block before the shift
        const int ic = i0 + c * 16;
        uint32_t w[4] = {0x88888888u, 0x88888888u, 0x88888888u, 0x88888888u};
        if (tr0 + t < nt) {
            const int cd = (vec_ok && ic + 16 <= N) ? sa.chunk_delay[ic >> 4] : -1;
            if (cd >= 0 && tt - cd >= 0) {
                const uint4 v = *reinterpret_cast<const uint4 *>(block + ((tt - cd) * F + f) * N + ic);
                w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
            } else {
                for (int m = 0; m < 16; m++) {
                    const int i = ic + m;
                    if (i >= N) break;
                    const int64_t src = tt - sa.delay[i];
                    const uint32_t byte = src >= 0 ? block[(src * F + f) * N + i]
                                                   : sa.hist[((sa.H + src) * F + f) * sa.S + sa.slot[i]];
                    w[m >> 2] = (w[m >> 2] & ~(0xFFu << (8 * (m & 3)))) | (byte << (8 * (m & 3)));
                }
            }
        }
        uint32_t *dst = tile + row_word(t) + c * 4;
        dst[0] = w[0]; dst[1] = w[1]; dst[2] = w[2]; dst[3] = w[3];
    }
    __syncthreads();
    decode_tile_store(tile, planes, t_pad, n_pad, tr0, i0, fl);
}

// Shift fix-up after a plain decode of samples t0 .. t0 + nt - 1: the plane
// rows of the S delayed inputs (inputs[s], delay d) are rewritten with the
// codes of x_i(t - d) -- from the block when t - d >= 0, else from the
// history -- leaving every other row (and the padding past nt) as decoded.
// One thread per (channel, delayed input, sample): writes are contiguous
// along the sample, and the gathers run with the whole GPU's parallelism.
__global__ void shift_fixup_kernel(const uint8_t *__restrict__ block, int64_t t0, int64_t nt, int32_t F, int32_t N,
                                   int32_t f0, int32_t nf, const ShiftArgs sa, const int32_t *__restrict__ inputs,
                                   uint8_t *__restrict__ planes, int64_t t_pad, int64_t n_pad)
{
    const int64_t total = (int64_t)nf * sa.S * nt;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = k % nt;
        const int32_t sl = (int32_t)((k / nt) % sa.S);
        const int64_t fl = k / (nt * sa.S);
        const int64_t f = f0 + fl;
        const int32_t i = inputs[sl];
        const int64_t src = t0 + t - sa.delay[i];
        const uint32_t byte = src >= 0 ? block[(src * F + f) * N + i] : sa.hist[((sa.H + src) * F + f) * sa.S + sl];
        const uint32_t codes = nib2_to_e4m3(byte | (byte << 12));  // low nibble -> byte 0, high nibble -> byte 1
        planes[((fl * 2 + 0) * n_pad + i) * t_pad + t] = (uint8_t)(codes >> 8);  // real part: high nibble
        planes[((fl * 2 + 1) * n_pad + i) * t_pad + t] = (uint8_t)(codes & 0xFFu);
    }
}

// History after a block of n samples, [H][F][S]: entry (h, f, s) is sample
// n - H + h of input inputs[s] -- from the block when that index is >= 0,
// else entry n + h of the old history.
__global__ void shift_history_kernel(const uint8_t *__restrict__ hist_old, const uint8_t *__restrict__ block,
                                     int64_t n, int32_t F, int32_t N, const int32_t *__restrict__ inputs, int32_t S,
                                     int64_t H, uint8_t *__restrict__ hist_new)
{
    const int64_t total = H * F * S;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t sl = (int32_t)(k % S);
        const int64_t f = (k / S) % F;
        const int64_t h = k / ((int64_t)S * F);
        const int64_t src = n - H + h;
        hist_new[k] = src >= 0 ? block[(src * F + f) * N + inputs[sl]] : hist_old[((n + h) * F + f) * S + sl];
    }
}

}  // namespace

cudaError_t launch_decode_shifted(const uint8_t *block, int64_t t0, int64_t nt, int32_t F, int32_t N, int32_t f0,
                                  int32_t nf, const ShiftArgs &sa, uint8_t *planes, int64_t t_pad, int64_t n_pad,
                                  cudaStream_t s)
{
    if (nf <= 0 || t_pad <= 0) return cudaSuccess;
    const int vec_ok = decode_vec_ok(block, N);
    dim3 grid((unsigned)(t_pad / 128), (unsigned)(n_pad / 128), (unsigned)nf);
    decode_shifted_kernel<<<grid, kDecThreads, 0, s>>>(block, t0, nt, F, N, f0, sa, planes, t_pad, n_pad, vec_ok);
    return cudaGetLastError();
}

cudaError_t launch_shift_fixup(const uint8_t *block, int64_t t0, int64_t nt, int32_t F, int32_t N, int32_t f0,
                               int32_t nf, const ShiftArgs &sa, const int32_t *inputs, uint8_t *planes, int64_t t_pad,
                               int64_t n_pad, cudaStream_t s)
{
    const int64_t total = (int64_t)nf * sa.S * nt;
    if (total <= 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    shift_fixup_kernel<<<(unsigned)blocks, 256, 0, s>>>(block, t0, nt, F, N, f0, nf, sa, inputs, planes, t_pad, n_pad);
    return cudaGetLastError();
}

cudaError_t launch_shift_history(const uint8_t *hist_old, const uint8_t *block, int64_t n, int32_t F, int32_t N,
                                 const int32_t *inputs, int32_t S, int64_t H, uint8_t *hist_new, cudaStream_t s)
{
    const int64_t total = H * F * S;
    if (total <= 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    shift_history_kernel<<<(unsigned)blocks, 256, 0, s>>>(hist_old, block, n, F, N, inputs, S, H, hist_new);
    return cudaGetLastError();
}

cudaError_t launch_decode(const uint8_t *block, int64_t T, int32_t F, int32_t N, int32_t f0,
                          int32_t nf, uint8_t *planes, int64_t t_pad, int64_t n_pad, cudaStream_t s)
{
    if (nf <= 0 || t_pad <= 0) return cudaSuccess;
    const int vec_ok = decode_vec_ok(block, N);
    dim3 grid((unsigned)(t_pad / 128), (unsigned)(n_pad / 128), (unsigned)nf);
    decode_kernel<<<grid, kDecThreads, 0, s>>>(block, T, F, N, f0, planes, t_pad, n_pad, vec_ok);
    return cudaGetLastError();
}

int decode_vec_ok(const uint8_t *block, int32_t N)
{
    return ((reinterpret_cast<uintptr_t>(block) & 15) == 0) && (N % 16 == 0);
}

cudaError_t launch_decode_batch(const DecodeJob *jobs, int n_jobs, int64_t total_ctas, cudaStream_t s)
{
    if (n_jobs <= 0 || total_ctas <= 0) return cudaSuccess;
    if (total_ctas > 2147483647LL) return cudaErrorInvalidValue;
    decode_batch_kernel<<<(unsigned)total_ctas, kDecThreads, 0, s>>>(jobs, n_jobs);
    return cudaGetLastError();
}

}  // namespace xeng

namespace xeng {

namespace {
__global__ void counts_finish_kernel(int32_t *__restrict__ counts, int dirty, const GateBase base, int32_t G,
                                     int64_t per_gate)
{
    const int64_t total = (int64_t)G * per_gate;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x)
        counts[k] = (dirty ? counts[k] : 0) + (int32_t)base.v[k / per_gate];
}
}  // namespace

cudaError_t launch_counts_finish(int32_t *counts, int dirty, const GateBase &base, int32_t G, int64_t per_gate,
                                 cudaStream_t s)
{
    if (G <= 0 || G > kMaxGates || per_gate <= 0) return cudaErrorInvalidValue;
    int64_t blocks = ((int64_t)G * per_gate + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    counts_finish_kernel<<<(unsigned)blocks, 256, 0, s>>>(counts, dirty, base, G, per_gate);
    return cudaGetLastError();
}

cudaError_t launch_decode_gather(const uint8_t *block, int32_t F, int32_t N, int32_t f0, int32_t nf, const int32_t *idx,
                                 int64_t Tg, const uint8_t *valid, uint8_t *planes, int64_t t_pad, int64_t n_pad,
                                 int32_t *counts, cudaStream_t s)
{
    if (nf <= 0 || t_pad <= 0) return cudaSuccess;
    dim3 grid((unsigned)(t_pad / 128), (unsigned)(n_pad / 128), (unsigned)nf);
    const int vec_ok = decode_vec_ok(block, N) && (!valid || (reinterpret_cast<uintptr_t>(valid) & 15) == 0);
    decode_gather_kernel<<<grid, kDecThreads, 0, s>>>(block, F, N, f0, idx, Tg, valid, planes, t_pad, n_pad, counts,
                                                      vec_ok);
    return cudaGetLastError();
}

}  // namespace xeng
