// nibble.cuh -- offset-nibble decode to FP8 E4M3 codes (paper Sec. II-A and
// its footnote: each 4-bit nibble stores value + 8, values in [-8, 7]; the
// high nibble is the real part, the low nibble the imaginary part; integers
// -8..7 are exact in E4M3).  Bulk paths use a table lookup in byte permutes;
// the half-precision route (a nibble u in the mantissa of 1024.0 gives
// 1024 + u, minus 1032 is u - 8, then the hardware converter) serves single
// bytes.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

namespace xeng {
namespace {

// Two offset nibbles (in bits 0-3 and 16-19 of x) to the half2 of their
// values u - 8.
__device__ __forceinline__ uint32_t nib2_lo_half2(uint32_t x)
{
    uint32_t v = (x & 0x000F000Fu) | 0x64006400u;  // half2(1024 + u_lo, 1024 + u_hi)
    __half2 hv = *reinterpret_cast<__half2 *>(&v);
    hv = __hsub2(hv, __halves2half2(__ushort_as_half(0x6408), __ushort_as_half(0x6408)));  // - 1032
    return *reinterpret_cast<uint32_t *>(&hv);
}

// The same for nibbles in bits 4-7 and 20-23, without shifting them down:
// they land in mantissa bits 4-7 (1024 + 16 u), and (1024 + 16 u) / 16 - 72 =
// u - 8, one exact half-precision FMA.
__device__ __forceinline__ uint32_t nib2_hi_half2(uint32_t x)
{
    uint32_t v = (x & 0x00F000F0u) | 0x64006400u;  // half2(1024 + 16 u_lo, 1024 + 16 u_hi)
    __half2 hv = *reinterpret_cast<__half2 *>(&v);
    hv = __hfma2(hv, __halves2half2(__ushort_as_half(0x2C00), __ushort_as_half(0x2C00)),   // x 1/16
                 __halves2half2(__ushort_as_half(0xD480), __ushort_as_half(0xD480)));  // - 72
    return *reinterpret_cast<uint32_t *>(&hv);
}

__device__ __forceinline__ uint32_t half2_to_e4m3x2(uint32_t v)
{
    __half2_raw h = *reinterpret_cast<__half2_raw *>(&v);
    return (uint32_t)__nv_cvt_halfraw2_to_fp8x2(h, __NV_SATFINITE, __NV_E4M3);
}

// Two offset nibbles (bits 0-3 and 16-19, or 4-7 and 20-23) to two E4M3 codes
// (bits 0-7 and 8-15 of the result).
__device__ __forceinline__ uint32_t nib2_to_e4m3(uint32_t x) { return half2_to_e4m3x2(nib2_lo_half2(x)); }
__device__ __forceinline__ uint32_t nib2_hi_to_e4m3(uint32_t x) { return half2_to_e4m3x2(nib2_hi_half2(x)); }

// Four offset nibbles (bits 0-15 of x, lowest first) to their four E4M3 codes
// by table lookup in byte permutes, without the conversion instruction (which
// issues at a fraction of the integer rate: on GB300 a decode with it ran at
// 0.83x the rate of this one, bit-identical over every 16-bit pattern).
// E4M3 codes of v = u - 8: for u >= 8 (v = 0..7) 00 38 40 44 48 4A 4C 4E; for
// u < 8 (v = -8..-1) D0 CE CC CA C8 C4 C0 B8, i.e. 0x80 | (50 4E 4C 4A 48 44 40
// 38).  Two permutes look up both tables by u & 7; a third, with each nibble
// as its selector, yields 0x7F where u < 8 and 0x00 where u >= 8 (a selector
// with bit 3 set replicates the sign of the picked byte, 0x7F: positive).
__device__ __forceinline__ uint32_t nib4_to_e4m3(uint32_t x)
{
    const uint32_t sel = x & 0x7777u;
    const uint32_t pos = __byte_perm(0x44403800u, 0x4E4C4A48u, sel);  // codes of 0..7
    const uint32_t neg = __byte_perm(0x4A4C4E50u, 0x38404448u, sel);  // codes of -8..-1 without the sign bit
    uint32_t m;
    asm("prmt.b32 %0, %1, %1, %2;" : "=r"(m) : "r"(0x7F7F7F7Fu), "r"(x));
    return (pos & ~m) | (neg & m) | ((m << 1) & 0x80808080u);
}

// Raw offset nibbles as FP6 E2M3 codes, without decoding: in E2M3 (sign, two
// exponent bits with bias 1, three mantissa bits) the subnormal binade and the
// first normal binade share the spacing 1/8, so the code whose low four bits
// are a nibble u (0..15) and whose top two bits are clear has the value u / 8
// exactly.  A product of two such operands is u u' / 64 and the offset
// (value = u - 8) is applied afterwards in integer arithmetic.  One word of
// four raw bytes (inputs 0..3 of one sample; high nibble Re, low nibble Im)
// gives the interleaved (Im, Re) codes of inputs 0, 1 and of inputs 2, 3.
__device__ __forceinline__ void raw4_to_e2m3_pairs(uint32_t w, uint32_t &c01, uint32_t &c23)
{
    const uint32_t lo = w & 0x0F0F0F0Fu;         // Im nibbles of inputs 0..3
    const uint32_t hi = (w >> 4) & 0x0F0F0F0Fu;  // Re nibbles of inputs 0..3
    c01 = __byte_perm(lo, hi, 0x5140);           // Im0 Re0 Im1 Re1
    c23 = __byte_perm(lo, hi, 0x7362);           // Im2 Re2 Im3 Re3
}

// Word of 4 samples (bytes = times t..t+3 of one input) -> (real codes, imag codes).
__device__ __forceinline__ void decode_word(uint32_t c, uint32_t &re, uint32_t &im)
{
    const uint32_t x01 = nib4_to_e4m3(c);        // [im0 re0 im1 re1]
    const uint32_t x23 = nib4_to_e4m3(c >> 16);  // [im2 re2 im3 re3]
    re = __byte_perm(x01, x23, 0x7531);
    im = __byte_perm(x01, x23, 0x6420);
}

// Transpose + decode of a 4 x 4 byte block: r[k] holds sample k of inputs
// 0..3 (byte m = input m); the result is input m's real and imaginary codes
// of samples 0..3.  A byte permute gathers input m of two samples into the
// low half of a word, whose four nibbles then go through the table at once.
__device__ __forceinline__ void decode_input4(const uint32_t r[4], int m, uint32_t &re, uint32_t &im)
{
    const uint32_t sel = (uint32_t)m | ((uint32_t)(4 + m) << 4);  // byte 0 <- first.m, byte 1 <- second.m
    const uint32_t x01 = nib4_to_e4m3(__byte_perm(r[0], r[1], sel));  // [im0 re0 im1 re1]
    const uint32_t x23 = nib4_to_e4m3(__byte_perm(r[2], r[3], sel));  // [im2 re2 im3 re3]
    re = __byte_perm(x01, x23, 0x7531);
    im = __byte_perm(x01, x23, 0x6420);
}

}  // namespace
}  // namespace xeng
