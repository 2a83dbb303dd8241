/* synth_host.c -- host side of the synthetic-data generators (synth_core.h). */
#include "synth_core.h"

uint64_t synth_key_c(uint64_t seed, uint64_t stream) { return synth_key(seed, stream); }

/* Bytes k0 .. k0+n-1 of the uniform stream `key`. */
void synth_uniform_host(uint8_t *out, int64_t n, uint64_t key, int64_t k0)
{
    #pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; k++)
        out[k] = synth_uniform_byte(key, (uint64_t)(k0 + k));
}

/* Sky-plus-noise block [T][F][N] restricted to times t0..t0+nt-1 and channels
 * f0..f0+nf-1; out is [nt][nf][N]. */
void synth_sky_host(uint8_t *out, int64_t t0, int64_t nt, int64_t f0, int64_t nf,
                    int64_t F, int64_t N, uint64_t key_s, uint64_t key_n,
                    int64_t cs, int64_t cn)
{
    #pragma omp parallel for schedule(static)
    for (int64_t tt = 0; tt < nt; tt++)
        for (int64_t ff = 0; ff < nf; ff++)
            for (int64_t i = 0; i < N; i++)
                out[(tt * nf + ff) * N + i] =
                    synth_sky_byte(key_s, key_n, cs, cn, t0 + tt, f0 + ff, i, F, N);
}
