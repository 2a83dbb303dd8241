/* synth_dev.cu -- device side of the synthetic-data generators (synth_core.h):
 * fills device buffers with exactly the bytes synth_host.c produces. */
#include <cuda_runtime.h>
#include "synth_core.h"

__global__ void synth_uniform_kernel(uint8_t *out, int64_t n, uint64_t key, int64_t k0)
{
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  /* one draw = 8 bytes */
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; w * 8 < n; w += stride) {
        for (int b = 0; b < 8; b++) {
            int64_t k = w * 8 + b;
            if (k < n) out[k] = synth_uniform_byte(key, (uint64_t)(k0 + k));
        }
    }
}

__global__ void synth_sky_kernel(uint8_t *out, int64_t T, int64_t F, int64_t N,
                                 uint64_t key_s, uint64_t key_n, int64_t cs, int64_t cn)
{
    int64_t total = T * F * N;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += stride) {
        int64_t i = k % N, tf = k / N;
        out[k] = synth_sky_byte(key_s, key_n, cs, cn, tf / F, tf % F, i, F, N);
    }
}

extern "C" int synth_uniform_dev(uint8_t *out, int64_t n, uint64_t key, int64_t k0, void *stream)
{
    if (n <= 0) return 0;
    synth_uniform_kernel<<<152 * 8, 256, 0, (cudaStream_t)stream>>>(out, n, key, k0);
    return (int)cudaGetLastError();
}

extern "C" int synth_sky_dev(uint8_t *out, int64_t T, int64_t F, int64_t N,
                             uint64_t key_s, uint64_t key_n, int64_t cs, int64_t cn, void *stream)
{
    if (T * F * N <= 0) return 0;
    synth_sky_kernel<<<152 * 8, 256, 0, (cudaStream_t)stream>>>(out, T, F, N, key_s, key_n, cs, cn);
    return (int)cudaGetLastError();
}
