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

// Two offset nibbles (in bits 0-3 and 16-19 of x) to two E4M3 codes.
__device__ __forceinline__ uint32_t nib2_to_e4m3(uint32_t x)
{
    __half2_raw h;
    uint32_t v = (x & 0x000F000Fu) | 0x64006400u;  // half2(1024 + u_lo, 1024 + u_hi)
    __half2 hv = *reinterpret_cast<__half2 *>(&v);
    hv = __hsub2(hv, __halves2half2(__ushort_as_half(0x6408), __ushort_as_half(0x6408)));  // - 1032
    h = *reinterpret_cast<__half2_raw *>(&hv);
    return (uint32_t)__nv_cvt_halfraw2_to_fp8x2(h, __NV_SATFINITE, __NV_E4M3);
}

// Word of 4 samples (bytes = times t..t+3 of one input) -> (real codes, imag codes).
__device__ __forceinline__ void decode_word(uint32_t c, uint32_t &re, uint32_t &im)
{
    uint32_t r02 = nib2_to_e4m3(c >> 4);   // high nibbles of bytes 0 and 2
    uint32_t r13 = nib2_to_e4m3(c >> 12);  // high nibbles of bytes 1 and 3
    uint32_t i02 = nib2_to_e4m3(c);        // low nibbles of bytes 0 and 2
    uint32_t i13 = nib2_to_e4m3(c >> 8);   // low nibbles of bytes 1 and 3
    re = __byte_perm(r02, r13, 0x5140);
    im = __byte_perm(i02, i13, 0x5140);
}

}  // namespace
}  // namespace xeng
