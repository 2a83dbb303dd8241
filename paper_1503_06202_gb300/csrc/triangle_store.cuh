// triangle_store.cuh -- the int32 triangle stores of the raw-nibble
// correlators' epilogues: eight (Re, Im) pairs of one row, stored or added
// in the widest pieces the row's alignment allows.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace xeng {
namespace {

// Store (kAdd false) or add (kAdd true) the 8 pairs (re[e], im[e]) at p[e]
// for e in [e_lo, e_hi) within [0, 8).  Whole chunks go out as 32-byte stores
// of four pairs (8- and 16-byte pieces at the ends by p's offset in a 32-byte
// sector), all loads before any store; the rest pair by pair.  Streaming
// accesses: the triangle is not read again here.
template <bool kAdd>
__device__ __forceinline__ void put8(int2 *p, int e_lo, int e_hi, const uint32_t (&re)[8],
                                     const uint32_t (&im)[8])
{
    if (e_lo <= 0 && e_hi >= 8) {
        uint32_t v[16];  // (re, im) interleaved, plus the old values when adding
        #pragma unroll
        for (int e = 0; e < 8; e++) {
            v[2 * e] = re[e];
            v[2 * e + 1] = im[e];
        }
        const int mis = (int)((reinterpret_cast<uintptr_t>(p) >> 3) & 3);  // pairs past a 32-byte boundary
        if (kAdd) {
            uint32_t o[16];
            auto ld8 = [&](int e) {
                const int2 x = __ldcs(p + e);
                o[2 * e] = (uint32_t)x.x;
                o[2 * e + 1] = (uint32_t)x.y;
            };
            auto ld16 = [&](int e) {
                const int4 x = __ldcs(reinterpret_cast<const int4 *>(p + e));
                o[2 * e] = (uint32_t)x.x;
                o[2 * e + 1] = (uint32_t)x.y;
                o[2 * e + 2] = (uint32_t)x.z;
                o[2 * e + 3] = (uint32_t)x.w;
            };
            auto ld32 = [&](int e) {
                asm volatile("ld.global.cs.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                             : "=r"(o[2 * e]), "=r"(o[2 * e + 1]), "=r"(o[2 * e + 2]), "=r"(o[2 * e + 3]),
                               "=r"(o[2 * e + 4]), "=r"(o[2 * e + 5]), "=r"(o[2 * e + 6]), "=r"(o[2 * e + 7])
                             : "l"(p + e));
            };
            switch (mis) {
                case 0: ld32(0); ld32(4); break;
                case 1: ld8(0); ld16(1); ld32(3); ld8(7); break;
                case 2: ld16(0); ld32(2); ld16(6); break;
                default: ld8(0); ld32(1); ld16(5); ld8(7); break;
            }
            #pragma unroll
            for (int k = 0; k < 16; k++) v[k] += o[k];
        }
        auto st8 = [&](int e) { __stcs(p + e, make_int2((int)v[2 * e], (int)v[2 * e + 1])); };
        auto st16 = [&](int e) {
            __stcs(reinterpret_cast<int4 *>(p + e),
                   make_int4((int)v[2 * e], (int)v[2 * e + 1], (int)v[2 * e + 2], (int)v[2 * e + 3]));
        };
        auto st32 = [&](int e) {
            asm volatile("st.global.cs.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                         ::"l"(p + e), "r"(v[2 * e]), "r"(v[2 * e + 1]), "r"(v[2 * e + 2]), "r"(v[2 * e + 3]),
                           "r"(v[2 * e + 4]), "r"(v[2 * e + 5]), "r"(v[2 * e + 6]), "r"(v[2 * e + 7])
                         : "memory");
        };
        switch (mis) {
            case 0: st32(0); st32(4); break;
            case 1: st8(0); st16(1); st32(3); st8(7); break;
            case 2: st16(0); st32(2); st16(6); break;
            default: st8(0); st32(1); st16(5); st8(7); break;
        }
    } else if (kAdd) {
        int2 old[8];
        #pragma unroll
        for (int e = 0; e < 8; e++)
            if (e >= e_lo && e < e_hi) old[e] = __ldcs(p + e);
        #pragma unroll
        for (int e = 0; e < 8; e++)
            if (e >= e_lo && e < e_hi) __stcs(p + e, make_int2(old[e].x + (int)re[e], old[e].y + (int)im[e]));
    } else {
        #pragma unroll
        for (int e = 0; e < 8; e++)
            if (e >= e_lo && e < e_hi) __stcs(p + e, make_int2((int)re[e], (int)im[e]));
    }
}

}  // namespace
}  // namespace xeng
