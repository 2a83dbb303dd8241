/*
 * oracle.c -- the X-engine oracle: a plain, slow, obviously correct CPU
 * correlator in int64.  TEST INFRASTRUCTURE ONLY: it is built, loaded and
 * called by the tests, by the smoke check and by the CPU-baseline leg of the
 * benchmark, never by the library.  It shares no code, header or table with
 * the CUDA path.
 *
 * What it computes (paper Sec. I and Sec. IV-C-1, "Full Correlation"; cost
 * in Eq. 1): for every frequency channel f and every input pair i <= j the
 * integrated visibility
 *
 *     V_ij(f) = sum_t x_i(t, f) * conj(x_j(t, f)),
 *
 * over all N(N+1)/2 pairs, autocorrelations i == j included (Eq. 1 counts
 * N(N+1)/2 products; 32,896 = 256*257/2 for the 256-input Pathfinder).
 *
 * Input format (Sec. II-A and its footnote): one byte per input per channel
 * per time sample; each 4-bit nibble stores value + 8, so values lie in
 * [-8, 7].  The high nibble is the real part, the low nibble the imaginary
 * part.  Layout [time][freq][input].
 *
 * Output: upper triangle, row-major, per channel contiguous:
 *     index(i, j) = i*N - i*(i-1)/2 + (j - i),  i <= j,
 * each entry (Re, Im) as int64 here (the caller narrows to int32 after
 * checking the bound).
 *
 * Since the method is exact integer arithmetic the oracle is the definition
 * itself: decode each sample, multiply, add -- nothing else.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Real and imaginary part of one offset-encoded 4+4-bit sample (Sec. II-A). */
static int64_t sample_re(uint8_t byte) { return (int64_t)(byte / 16) - 8; }
static int64_t sample_im(uint8_t byte) { return (int64_t)(byte % 16) - 8; }

static int64_t tri_index(int64_t i, int64_t j, int64_t n)
{
    return i * n - i * (i - 1) / 2 + (j - i);
}

/* Decode channel f of the block into int64 arrays re[i*T + t], im[i*T + t]. */
static void decode_channel(const uint8_t *in, int64_t T, int32_t F, int32_t N,
                           int32_t f, int64_t *re, int64_t *im)
{
    for (int64_t t = 0; t < T; t++)
        for (int64_t i = 0; i < N; i++) {
            uint8_t byte = in[(t * F + f) * (int64_t)N + i];
            re[i * T + t] = sample_re(byte);
            im[i * T + t] = sample_im(byte);
        }
}

/*
 * oracle_correlate: channels f0 .. f0+nf-1 of the block in[T][F][N].
 * out: int64 [nf][N(N+1)/2][2].  Returns 0, or -1 on bad arguments / no memory.
 */
int oracle_correlate(const uint8_t *in, int64_t T, int32_t F, int32_t N,
                     int32_t f0, int32_t nf, int64_t *out)
{
    if (T < 0 || F < 1 || N < 1 || f0 < 0 || nf < 0 || f0 + nf > F)
        return -1;
    int64_t nb = (int64_t)N * (N + 1) / 2;
    int64_t *re = malloc(sizeof(int64_t) * (size_t)(N * T + 1));
    int64_t *im = malloc(sizeof(int64_t) * (size_t)(N * T + 1));
    if (!re || !im) { free(re); free(im); return -1; }
    for (int32_t c = 0; c < nf; c++) {
        decode_channel(in, T, F, N, f0 + c, re, im);
        int64_t *o = out + (int64_t)c * nb * 2;
        #pragma omp parallel for schedule(dynamic, 1)
        for (int64_t i = 0; i < N; i++) {
            for (int64_t j = i; j < N; j++) {
                const int64_t *ar = re + i * T, *ai = im + i * T;
                const int64_t *br = re + j * T, *bi = im + j * T;
                int64_t vr = 0, vi = 0;
                for (int64_t t = 0; t < T; t++) {
                    /* (ar + i ai) * (br - i bi) */
                    vr += ar[t] * br[t] + ai[t] * bi[t];
                    vi += ai[t] * br[t] - ar[t] * bi[t];
                }
                int64_t k = tri_index(i, j, N);
                o[2 * k] = vr;
                o[2 * k + 1] = vi;
            }
        }
    }
    free(re);
    free(im);
    return 0;
}

/*
 * oracle_correlate_full: every ordered pair (i, j), lower triangle included,
 * each computed on its own from the definition.  out: int64 [nf][N][N][2].
 * Used to check Hermitian symmetry of the definition as implemented.
 */
int oracle_correlate_full(const uint8_t *in, int64_t T, int32_t F, int32_t N,
                          int32_t f0, int32_t nf, int64_t *out)
{
    if (T < 0 || F < 1 || N < 1 || f0 < 0 || nf < 0 || f0 + nf > F)
        return -1;
    for (int32_t c = 0; c < nf; c++) {
        int64_t *o = out + (int64_t)c * N * N * 2;
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; i++)
            for (int64_t j = 0; j < N; j++) {
                int64_t vr = 0, vi = 0;
                for (int64_t t = 0; t < T; t++) {
                    uint8_t x = in[(t * F + f0 + c) * (int64_t)N + i];
                    uint8_t y = in[(t * F + f0 + c) * (int64_t)N + j];
                    vr += sample_re(x) * sample_re(y) + sample_im(x) * sample_im(y);
                    vi += sample_im(x) * sample_re(y) - sample_re(x) * sample_im(y);
                }
                o[2 * (i * N + j)] = vr;
                o[2 * (i * N + j) + 1] = vi;
            }
    }
    return 0;
}

/*
 * oracle_correlate_pairs: V_ij(f) for a list of (f, i, j) triples, straight
 * from the definition (strided reads, no decode buffer).  Lets a test check
 * sampled outputs of a workload far too large for the full oracle.
 * out: int64 [n][2].
 */
int oracle_correlate_pairs(const uint8_t *in, int64_t T, int32_t F, int32_t N,
                           int64_t n, const int32_t *fs, const int32_t *is,
                           const int32_t *js, int64_t *out)
{
    if (T < 0 || F < 1 || N < 1 || n < 0)
        return -1;
    for (int64_t p = 0; p < n; p++)
        if (fs[p] < 0 || fs[p] >= F || is[p] < 0 || is[p] >= N || js[p] < 0 || js[p] >= N)
            return -1;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < n; p++) {
        int64_t vr = 0, vi = 0;
        for (int64_t t = 0; t < T; t++) {
            uint8_t x = in[(t * F + fs[p]) * (int64_t)N + is[p]];
            uint8_t y = in[(t * F + fs[p]) * (int64_t)N + js[p]];
            vr += sample_re(x) * sample_re(y) + sample_im(x) * sample_im(y);
            vi += sample_im(x) * sample_re(y) - sample_re(x) * sample_im(y);
        }
        out[2 * p] = vr;
        out[2 * p + 1] = vi;
    }
    return 0;
}

/*
 * oracle_beam_power: the left-hand side of the weighted-sum identity
 *     sum_t |sum_i w_i x_i(t)|^2 = sum_{i,j} w_i conj(w_j) V_ij,
 * per channel, for Gaussian-integer weights w (w_re[i] + i w_im[i]).
 * O(N T) per channel; it never forms a product of two inputs' samples, so it
 * checks a correlator output without re-running the pair loop.
 * out: int64 [nf].
 */
int oracle_beam_power(const uint8_t *in, int64_t T, int32_t F, int32_t N,
                      int32_t f0, int32_t nf, const int64_t *w_re,
                      const int64_t *w_im, int64_t *out)
{
    if (T < 0 || F < 1 || N < 1 || f0 < 0 || nf < 0 || f0 + nf > F)
        return -1;
    #pragma omp parallel for schedule(static)
    for (int32_t c = 0; c < nf; c++) {
        int64_t acc = 0;
        for (int64_t t = 0; t < T; t++) {
            int64_t sr = 0, si = 0;
            for (int64_t i = 0; i < N; i++) {
                uint8_t x = in[(t * F + f0 + c) * (int64_t)N + i];
                int64_t xr = sample_re(x), xi = sample_im(x);
                sr += w_re[i] * xr - w_im[i] * xi;
                si += w_re[i] * xi + w_im[i] * xr;
            }
            acc += sr * sr + si * si;
        }
        out[c] = acc;
    }
    return 0;
}

/* Number of OpenMP threads the oracle's parallel loops use (1 without OpenMP). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * oracle_correlate_gated: gating (Sec. IV-C-4: the integration is split into
 * sub-buffers by the time of each sample relative to a source's period) and
 * flagged data (Sec. IV-A: missing or saturated samples are tracked and their
 * count is reported for renormalising the integrated matrices).
 *
 * gate[t] in [0, G) names the sub-buffer sample t goes to; any other value
 * drops the sample.  valid[t][f][i] != 0 marks a usable sample; NULL means
 * every sample is usable.  For every gate g, channel f and pair i <= j:
 *
 *     V^g_ij(f) = sum over t with gate[t] == g, valid_i(t), valid_j(t)
 *                 of x_i(t, f) * conj(x_j(t, f)),
 *     counts[g][f][i] = number of t with gate[t] == g and valid_i(t).
 *
 * out: int64 [G][F][N(N+1)/2][2]; counts: int64 [G][F][N] or NULL.
 */
int oracle_correlate_gated(const uint8_t *in, int64_t T, int32_t F, int32_t N, const int32_t *gate, int32_t G,
                           const uint8_t *valid, int64_t *out, int64_t *counts)
{
    if (T < 0 || F < 1 || N < 1 || G < 1 || !gate)
        return -1;
    const int64_t nb = (int64_t)N * (N + 1) / 2;
    memset(out, 0, sizeof(int64_t) * (size_t)(G * F * nb * 2));
    if (counts)
        memset(counts, 0, sizeof(int64_t) * (size_t)(G * F * N));
    for (int32_t f = 0; f < F; f++) {
        #pragma omp parallel for schedule(dynamic, 1)
        for (int64_t i = 0; i < N; i++) {
            for (int64_t t = 0; t < T; t++) {
                const int32_t g = gate[t];
                if (g < 0 || g >= G) continue;
                const int64_t at = (t * F + f) * (int64_t)N;
                if (valid && !valid[at + i]) continue;
                if (counts) counts[((int64_t)g * F + f) * N + i] += 1;
                const uint8_t x = in[at + i];
                int64_t *o = out + ((int64_t)g * F + f) * nb * 2;
                for (int64_t j = i; j < N; j++) {
                    if (valid && !valid[at + j]) continue;
                    const uint8_t y = in[at + j];
                    const int64_t k = tri_index(i, j, N);
                    o[2 * k] += sample_re(x) * sample_re(y) + sample_im(x) * sample_im(y);
                    o[2 * k + 1] += sample_im(x) * sample_re(y) - sample_re(x) * sample_im(y);
                }
            }
        }
    }
    return 0;
}

/*
 * oracle_correlate_shifted: time shifting (Sec. IV-C-5: an input from an
 * outlying station is delayed inside the correlator so that its signal lines
 * up with the others again).  Input i is delayed by delays[i] >= 0 samples:
 *
 *     y_i(t, f) = x_i(t - delays[i], f),  and 0 where t - delays[i] < 0
 *
 * (nothing precedes the stream's first sample).  For the window
 * t_a <= t < t_b of the stream in[T][F][N] and every channel f, pair i <= j:
 *
 *     V_ij(f) = sum_{t = t_a}^{t_b - 1} y_i(t, f) * conj(y_j(t, f)).
 *
 * out: int64 [F][N(N+1)/2][2].  Returns 0, or -1 on bad arguments / no memory.
 */
int oracle_correlate_shifted(const uint8_t *in, int64_t T, int32_t F, int32_t N, const int32_t *delays, int64_t t_a,
                             int64_t t_b, int64_t *out)
{
    if (T < 0 || F < 1 || N < 1 || !delays || t_a < 0 || t_b < t_a || t_b > T)
        return -1;
    for (int32_t i = 0; i < N; i++)
        if (delays[i] < 0)
            return -1;
    const int64_t W = t_b - t_a, nb = (int64_t)N * (N + 1) / 2;
    int64_t *re = malloc(sizeof(int64_t) * (size_t)(N * W + 1));
    int64_t *im = malloc(sizeof(int64_t) * (size_t)(N * W + 1));
    if (!re || !im) { free(re); free(im); return -1; }
    for (int32_t f = 0; f < F; f++) {
        /* the delayed series y_i over the window */
        for (int64_t i = 0; i < N; i++)
            for (int64_t w = 0; w < W; w++) {
                const int64_t s = t_a + w - delays[i];
                re[i * W + w] = s >= 0 ? sample_re(in[(s * F + f) * (int64_t)N + i]) : 0;
                im[i * W + w] = s >= 0 ? sample_im(in[(s * F + f) * (int64_t)N + i]) : 0;
            }
        int64_t *o = out + (int64_t)f * nb * 2;
        #pragma omp parallel for schedule(dynamic, 1)
        for (int64_t i = 0; i < N; i++)
            for (int64_t j = i; j < N; j++) {
                int64_t vr = 0, vi = 0;
                for (int64_t w = 0; w < W; w++) {
                    vr += re[i * W + w] * re[j * W + w] + im[i * W + w] * im[j * W + w];
                    vi += im[i * W + w] * re[j * W + w] - re[i * W + w] * im[j * W + w];
                }
                o[2 * tri_index(i, j, N)] = vr;
                o[2 * tri_index(i, j, N) + 1] = vi;
            }
    }
    free(re);
    free(im);
    return 0;
}

/*
 * oracle_beamform: discrete beamforming (Sec. IV-C-3: the data of all inputs
 * are phase-shifted and summed, which points a beam at a chosen sky direction;
 * the beam is written out at the full sample cadence).  With Gaussian-integer
 * weights w_{f,b,i} = w_re + i w_im, for every sample t, channel f, beam b:
 *
 *     y_b(t, f) = sum_i w_{f,b,i} * x_i(t, f).
 *
 * w_re, w_im: int32 [F][B][N].  out: int64 [T][F][B][2].
 */
int oracle_beamform(const uint8_t *in, int64_t T, int32_t F, int32_t N, const int32_t *w_re, const int32_t *w_im,
                    int32_t B, int64_t *out)
{
    if (T < 0 || F < 1 || N < 1 || B < 1 || !w_re || !w_im)
        return -1;
    #pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < T; t++)
        for (int64_t f = 0; f < F; f++)
            for (int64_t b = 0; b < B; b++) {
                int64_t yr = 0, yi = 0;
                for (int64_t i = 0; i < N; i++) {
                    const uint8_t x = in[(t * F + f) * (int64_t)N + i];
                    const int64_t wr = w_re[(f * B + b) * N + i], wi = w_im[(f * B + b) * N + i];
                    /* (wr + i wi) (xr + i xi) */
                    yr += wr * sample_re(x) - wi * sample_im(x);
                    yi += wr * sample_im(x) + wi * sample_re(x);
                }
                out[((t * F + f) * B + b) * 2] = yr;
                out[((t * F + f) * B + b) * 2 + 1] = yi;
            }
    return 0;
}
