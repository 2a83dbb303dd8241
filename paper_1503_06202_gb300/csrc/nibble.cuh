// nibble.cuh -- offset-nibble decode to FP8 E4M3 codes (paper Sec. II-A and
// its footnote: each 4-bit nibble stores value + 8, values in [-8, 7]; the
// high nibble is the real part, the low nibble the imaginary part).  A nibble
// u placed in the mantissa of the half 1024.0 gives 1024 + u; subtracting
// 1032 leaves u - 8 exactly, which the hardware converter packs to E4M3
// (integers -8..7 are exact there).
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

// Word of 4 samples (bytes = times t..t+3 of one input) -> (real codes, imag codes).
__device__ __forceinline__ void decode_word(uint32_t c, uint32_t &re, uint32_t &im)
{
    const uint32_t c8 = c >> 8;
    const uint32_t r02 = nib2_hi_to_e4m3(c);   // high nibbles of bytes 0 and 2
    const uint32_t r13 = nib2_hi_to_e4m3(c8);  // high nibbles of bytes 1 and 3
    const uint32_t i02 = nib2_to_e4m3(c);      // low nibbles of bytes 0 and 2
    const uint32_t i13 = nib2_to_e4m3(c8);     // low nibbles of bytes 1 and 3
    re = __byte_perm(r02, r13, 0x5140);
    im = __byte_perm(i02, i13, 0x5140);
}

// Transpose + decode of a 4 x 4 byte block: r[k] holds sample k of inputs
// 0..3 (byte m = input m); the result is input m's real and imaginary codes
// of samples 0..3.  One byte permute gathers input m of two samples into the
// two half lanes, so no separate transpose is needed.
__device__ __forceinline__ void decode_input4(const uint32_t r[4], int m, uint32_t &re, uint32_t &im)
{
    const uint32_t sel = (uint32_t)m | ((uint32_t)(4 + m) << 8);  // byte 0 <- first.m, byte 2 <- second.m
    const uint32_t p01 = __byte_perm(r[0], r[1], sel);
    const uint32_t p23 = __byte_perm(r[2], r[3], sel);
    re = __byte_perm(nib2_hi_to_e4m3(p01), nib2_hi_to_e4m3(p23), 0x5410);
    im = __byte_perm(nib2_to_e4m3(p01), nib2_to_e4m3(p23), 0x5410);
}

}  // namespace
}  // namespace xeng
