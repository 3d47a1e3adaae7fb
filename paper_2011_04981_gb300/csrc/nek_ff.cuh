// Float-float helpers shared by the FP64-accurate operator and the CG's dot
// products: a double split into an unevaluated pair of floats, and the pair
// joined back, with integer operations (the FP64 <-> FP32 conversion
// instructions run on GB300's FP64 pipe, 2 per SM per clock).
#pragma once

#include <cuda_runtime.h>

namespace nek {

// x = h + l with h = x truncated to 24 significant bits and l the next 23 bits
// (relative error <= 2^-46), built from the bit pattern with integer operations
// only: on GB300 the FP64<->FP32 conversion instructions share the FP64 pipe
// (2 per SM per clock), which this avoids.  Valid for 2^-80 <= |x| < 2^127
// (smaller magnitudes give l = 0, or h = l = 0 below 2^-126).
__device__ __forceinline__ float2 split_double(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sgn = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    // sign | (e - 896) << 23 | top 23 mantissa bits
    const unsigned hb = sgn | ((unsigned)(e - 896) << 23) | (((hi & 0xFFFFFu) << 3) | (lo >> 29));
    // next 23 mantissa bits (bits 6..28 of lo) as an integer, times 2^(e - 1069)
    const float r = __fsub_rn(__uint_as_float(0x4B000000u | ((lo >> 6) & 0x7FFFFFu)), 8388608.0f);
    const float l = __fmul_rn(r, __uint_as_float((unsigned)(e - 942) << 23));
    const float h = e >= 897 ? __uint_as_float(hb) : 0.0f;
    return make_float2(h, e >= 943 ? __uint_as_float(__float_as_uint(l) | sgn) : 0.0f);
}

// (double)h + (double)l with the two widenings done by integer operations and a
// single FP64 add.
__device__ __forceinline__ double widen(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned a = u & 0x7FFFFFFFu;
    if (a < 0x00800000u) return 0.0;  // zero or FP32-denormal: below the kernel's accuracy scale
    const unsigned hi = (u & 0x80000000u) | ((((a >> 23) + 896u) << 20) | ((a & 0x7FFFFFu) >> 3));
    const unsigned lo = (a & 0x7u) << 29;
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}
__device__ __forceinline__ double join_pair(float h, float l) { return __dadd_rn(widen(h), widen(l)); }

}  // namespace nek
