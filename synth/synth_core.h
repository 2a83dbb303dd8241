/*
 * synth_core.h -- seeded, counter-based generators of synthetic F-engine
 * data (4+4-bit offset-encoded complex samples, layout [time][freq][input]).
 *
 * This header holds no correlator arithmetic: it only makes input bytes.  It
 * is compiled twice, by gcc for the host (synth_host.c) and by nvcc for the
 * device (synth_dev.cu), so that both produce the same bytes for the same
 * seed; only integer operations are used, so the two agree bit for bit.
 *
 * Random source: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used counter-style:
 * draw(key, c) = mix64(key + (c + 1) * 0x9E3779B97F4A7C15).
 *
 * Normal variates: the Irwin-Hall sum of twelve uniforms minus six (mean 0,
 * variance 1), in 16-bit fixed point.
 */
#ifndef SYNTH_CORE_H
#define SYNTH_CORE_H
#include <stdint.h>

#ifdef __CUDACC__
#define SYNTH_HD static __host__ __device__ __forceinline__
#else
#define SYNTH_HD static inline
#endif

#define SYNTH_GAMMA 0x9E3779B97F4A7C15ULL

SYNTH_HD uint64_t synth_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

SYNTH_HD uint64_t synth_draw(uint64_t key, uint64_t c)
{
    return synth_mix64(key + (c + 1) * SYNTH_GAMMA);
}

/* Key of sub-stream `stream` under master seed `seed` (jobs, channels, ...). */
SYNTH_HD uint64_t synth_key(uint64_t seed, uint64_t stream)
{
    return synth_draw(synth_draw(0, seed), stream);
}

/* Uniform bytes: byte k of the block is byte (k mod 8) of draw(key, k / 8). */
SYNTH_HD uint8_t synth_uniform_byte(uint64_t key, uint64_t k)
{
    return (uint8_t)(synth_draw(key, k >> 3) >> (8 * (k & 7)));
}

/* N(0,1) in units of 2^-16: sum of twelve 16-bit uniforms minus 6 * 2^16,
 * from draws c0, c0+1, c0+2. */
SYNTH_HD int64_t synth_normal_q16(uint64_t key, uint64_t c0)
{
    int64_t s = 0;
    for (int d = 0; d < 3; d++) {
        uint64_t r = synth_draw(key, c0 + d);
        s += (int64_t)(r & 0xFFFF) + (int64_t)((r >> 16) & 0xFFFF)
           + (int64_t)((r >> 32) & 0xFFFF) + (int64_t)(r >> 48);
    }
    return s - 6 * 65536;
}

/* One 4-bit component: x = cs*s + cn*n (2^-32 units), rounded half away from
 * zero, clipped to [-8, 7], stored as value + 8. */
SYNTH_HD uint32_t synth_component(int64_t s_q16, int64_t n_q16, int64_t cs, int64_t cn)
{
    int64_t x = cs * s_q16 + cn * n_q16;
    int64_t mag = ((x < 0 ? -x : x) + ((int64_t)1 << 31)) >> 32;
    int64_t q = x < 0 ? -mag : mag;
    if (q < -8) q = -8;
    if (q > 7) q = 7;
    return (uint32_t)(q + 8);
}

/*
 * Sky-plus-noise byte for (t, f, i): per real component a shared term s (one
 * per (t, f), common to all inputs) and an independent term n (per input),
 * x = sigma (sqrt(rho) s + sqrt(1 - rho) n); cs = round(sigma sqrt(rho) 2^16),
 * cn = round(sigma sqrt(1 - rho) 2^16).  key_s and key_n are the two streams.
 */
SYNTH_HD uint8_t synth_sky_byte(uint64_t key_s, uint64_t key_n, int64_t cs, int64_t cn,
                                int64_t t, int64_t f, int64_t i, int64_t F, int64_t N)
{
    uint64_t cs0 = (uint64_t)(t * F + f) * 6;
    uint64_t cn0 = (uint64_t)((t * F + f) * N + i) * 6;
    uint32_t re = synth_component(synth_normal_q16(key_s, cs0), synth_normal_q16(key_n, cn0), cs, cn);
    uint32_t im = synth_component(synth_normal_q16(key_s, cs0 + 3), synth_normal_q16(key_n, cn0 + 3), cs, cn);
    return (uint8_t)((re << 4) | im);
}

#endif
