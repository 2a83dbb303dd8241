// correlate_dp4a.cu -- the plain CUDA-core correlator: the same visibilities
// (paper Sec. IV-C-1, Eq. 1) computed with int8 dot products (dp4a) and int32
// accumulators, straight from the 4+4-bit bytes.  It is the per-instance
// comparison kernel for the tensor engine and needs no decode buffer.
//
// Per 2 samples an input's values pack into one word x = [a_t, b_t, a_t+1, b_t+1]
// (a = Re, b = Im, int8), and for the conjugated side also y = [-b_t, a_t,
// -b_t+1, a_t+1].  Then dp4a(x_i, x_j) = sum (a_i a_j + b_i b_j) = Re V_ij
// and dp4a(x_i, y_j) = sum (b_i a_j - a_i b_j) = Im V_ij over the two samples.
//
// CTA = one channel x one 64 x 64 upper-triangle tile pair; 256 threads, each
// owns 4 x 4 (i, j) pairs; 32-sample chunks staged and decoded in shared memory.
#include "xeng_internal.h"

namespace xeng {
namespace {

constexpr int kDT = 64;   // inputs per tile side
constexpr int kDS = 32;   // samples per chunk

__device__ __forceinline__ uint32_t pack4(int v0, int v1, int v2, int v3)
{
    return (uint32_t)(v0 & 0xFF) | ((uint32_t)(v1 & 0xFF) << 8) | ((uint32_t)(v2 & 0xFF) << 16) |
           ((uint32_t)(v3 & 0xFF) << 24);
}

__global__ void __launch_bounds__(256)
correlate_dp4a_kernel(const uint8_t *__restrict__ block, int64_t T, int32_t F, int32_t N, int nt,
                      int32_t *__restrict__ acc, int accumulate)
{
    __shared__ uint8_t rawb[2][kDS][kDT];
    __shared__ __align__(16) uint32_t xs[2][kDS / 2][kDT];  // [0] = x of tile I, [1] = x of tile J
    __shared__ __align__(16) uint32_t ys[kDS / 2][kDT];     // y (conjugate side) of tile J

    int r = blockIdx.x, I = 0;
    while (r >= nt - I) { r -= nt - I; ++I; }
    const int J = I + r;
    const int64_t f = blockIdx.y;
    const int tid = threadIdx.x;
    const int ti = tid >> 4, tj = tid & 15;

    int accr[4][4], acci[4][4];
    #pragma unroll
    for (int x = 0; x < 4; x++)
        #pragma unroll
        for (int y = 0; y < 4; y++) accr[x][y] = acci[x][y] = 0;

    for (int64_t t0 = 0; t0 < T; t0 += kDS) {
        // stage raw bytes of both tiles; 0x88 (value 0 + 0i) outside the block
        for (int k = tid; k < 2 * kDS * kDT; k += 256) {
            const int sel = k / (kDS * kDT), rem = k % (kDS * kDT);
            const int t = rem / kDT, c = rem % kDT;
            const int64_t i = (int64_t)(sel ? J : I) * kDT + c;
            const int64_t tt = t0 + t;
            rawb[sel][t][c] = (tt < T && i < N) ? block[(tt * F + f) * N + i] : (uint8_t)0x88;
        }
        __syncthreads();
        for (int k = tid; k < 2 * (kDS / 2) * kDT; k += 256) {
            const int sel = k / ((kDS / 2) * kDT), rem = k % ((kDS / 2) * kDT);
            const int tp = rem / kDT, c = rem % kDT;
            const int b0 = rawb[sel][2 * tp][c], b1 = rawb[sel][2 * tp + 1][c];
            const int a0 = (b0 >> 4) - 8, i0 = (b0 & 15) - 8, a1 = (b1 >> 4) - 8, i1 = (b1 & 15) - 8;
            xs[sel][tp][c] = pack4(a0, i0, a1, i1);
            if (sel) ys[tp][c] = pack4(-i0, a0, -i1, a1);
        }
        __syncthreads();
        #pragma unroll 4
        for (int tp = 0; tp < kDS / 2; tp++) {
            const uint4 av = *reinterpret_cast<const uint4 *>(&xs[0][tp][ti * 4]);
            const uint4 bv = *reinterpret_cast<const uint4 *>(&xs[1][tp][tj * 4]);
            const uint4 cv = *reinterpret_cast<const uint4 *>(&ys[tp][tj * 4]);
            const int ax[4] = {(int)av.x, (int)av.y, (int)av.z, (int)av.w};
            const int bx[4] = {(int)bv.x, (int)bv.y, (int)bv.z, (int)bv.w};
            const int cx[4] = {(int)cv.x, (int)cv.y, (int)cv.z, (int)cv.w};
            #pragma unroll
            for (int x = 0; x < 4; x++)
                #pragma unroll
                for (int y = 0; y < 4; y++) {
                    accr[x][y] = __dp4a(ax[x], bx[y], accr[x][y]);
                    acci[x][y] = __dp4a(ax[x], cx[y], acci[x][y]);
                }
        }
        __syncthreads();
    }

    const int64_t n = N;
    int2 *out = reinterpret_cast<int2 *>(acc + f * n * (n + 1));
    #pragma unroll
    for (int x = 0; x < 4; x++) {
        const int64_t i = (int64_t)I * kDT + ti * 4 + x;
        if (i >= n) continue;
        const int64_t row_base = i * n - i * (i - 1) / 2 - i;
        #pragma unroll
        for (int y = 0; y < 4; y++) {
            const int64_t j = (int64_t)J * kDT + tj * 4 + y;
            if (j < i || j >= n) continue;
            int2 *p = out + row_base + j;
            if (accumulate) {
                const int2 o = *p;
                *p = make_int2(o.x + accr[x][y], o.y + acci[x][y]);
            } else {
                *p = make_int2(accr[x][y], acci[x][y]);
            }
        }
    }
}

}  // namespace

cudaError_t launch_correlate_dp4a(const uint8_t *block, int64_t T, int32_t F, int32_t N, int32_t *acc,
                                  int32_t accumulate, cudaStream_t s)
{
    const int nt = (N + kDT - 1) / kDT;
    const int pairs = nt * (nt + 1) / 2;
    for (int32_t f0 = 0; f0 < F; f0 += 65535) {
        const int32_t nf = (F - f0) < 65535 ? (F - f0) : 65535;
        dim3 grid((unsigned)pairs, (unsigned)nf);
        const int64_t nb2 = (int64_t)N * (N + 1);
        correlate_dp4a_kernel<<<grid, 256, 0, s>>>(block + (int64_t)f0 * N, T, F, N, nt, acc + f0 * nb2,
                                                   accumulate);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace xeng
