/*
 * xeng_peaks.h -- dense-throughput probes (part of libxeng.so) that measure
 * the roofline denominators for the correlator on the GPU at hand.
 *
 * The paper's cost measure is complex multiply-accumulates, Eq. 1, at 8 real
 * operations each (Sec. II: 4 TFLOPS ~ 0.5 TcMAC/s); these probes give the
 * dense rate of each instruction family the correlator could run on, as
 * TFLOP/s with 2 flops per multiply-add.
 */
#ifndef XENG_PEAKS_H
#define XENG_PEAKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#ifndef XENG_API
#define XENG_API __attribute__((visibility("default")))
#endif

#define XENG_PEAK_TC_F8F6F4   0  /* tcgen05.mma kind::f8f6f4, E4M3, M128 N256 K32, f32 accumulate */
#define XENG_PEAK_TC_F16      1  /* tcgen05.mma kind::f16, M128 N256 K16, f32 accumulate          */
#define XENG_PEAK_MMA_SYNC_S8 2  /* warp mma.sync m16n8k32 s8 x s8 -> s32 (legacy INT8 tensor)   */
#define XENG_PEAK_DP4A        3  /* CUDA-core dp4a (4 int8 products per instruction)             */
#define XENG_PEAK_TC_F8F6F4_N128 4  /* as XENG_PEAK_TC_F8F6F4 with N = 128                       */
#define XENG_PEAK_TC_F8F6F4_LIVE 6  /* as XENG_PEAK_TC_F8F6F4 with random codes of -8..7 instead of
                                       zeros (the power the tensor core draws depends on the data) */
#define XENG_PEAK_TC_F8F6F4_MIX  5  /* the correlator's mix per K step: one N = 256 and two N = 128
                                       (second with A negated) into one 256-column accumulator   */
#define XENG_PEAK_TC_F8F6F4_LIVE_RAW 7  /* as XENG_PEAK_TC_F8F6F4_LIVE with random raw-nibble codes
                                           (bytes 0x00..0x0F: E4M3 of u / 512)                    */
#define XENG_PEAK_TC_F8F6F4_MN 8    /* as XENG_PEAK_TC_F8F6F4_LIVE_RAW with both operands MN-major
                                       (128-byte swizzle; B two 128-element atoms along N)        */
#define XENG_PEAK_TC_F8F6F4_MN_N128 9  /* as XENG_PEAK_TC_F8F6F4_MN with N = 128                 */
#define XENG_PEAK_TC_F8F6F4_MN_RING 10 /* as XENG_PEAK_TC_F8F6F4_MN in the single-pass kernels'
                                          issue pattern: per 64-sample stage eight N = 256 MMAs into
                                          two accumulators (one with A negated), a commit to the
                                          stage's mbarrier, and a wait for the stage four back      */
#define XENG_PEAK_TC_F8F6F4_MN_PAIRS 11 /* the MMAs of XENG_PEAK_TC_F8F6F4_MN_RING without the ring:
                                           one commit at the end                                    */

/*
 * xeng_peak_probe -- run probe `kind` with `iters` instructions per issuing
 *   thread (one CTA per SM for tcgen05; several per SM otherwise) on the
 *   current device and legacy default stream; on success write the dense
 *   TFLOP/s to *tflops and the timed kernel's milliseconds to *ms.
 *   Synchronous.  Returns 0, -1 (bad argument), -4 (no memory), -5 (CUDA
 *   error) or -6 (a device-side wait timed out).  Allocates a 4-byte flag.
 */
XENG_API int xeng_peak_probe(int32_t kind, int64_t iters, double *tflops, double *ms);

#ifdef __cplusplus
}
#endif
#endif
