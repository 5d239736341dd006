// Conversions between binary32 and binary64 built from the IEEE-754 bit fields (binary32:
// sign, 8 exponent bits biased by 127, 23 fraction bits; binary64: sign, 11 exponent bits
// biased by 1023, 52 fraction bits), on the integer pipe.  On this GPU the conversion
// instructions issue at the FP64 pipe's rate (1/64 of FP32), so a phase that converts once or
// twice per node is bound by them; these run at more than twice that rate and leave the FP64
// pipe to the fp64 arithmetic.  Branch-free (selects only), so that no fallback conversion
// is predicated into the code.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace usfft {

// exact float -> double; zero and subnormal inputs give a signed zero, inf and nan keep their class
__device__ __forceinline__ double f2d_exact(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    const uint32_t de = e == 0 ? 0u : (e == 255u ? 2047u : e + 896u);
    const uint32_t hi = (b & 0x80000000u) | (de << 20) | (e == 0 ? 0u : ((b >> 3) & 0xfffffu));
    const uint32_t lo = e == 0 ? 0u : (b << 29);
    return __hiloint2double((int)hi, (int)lo);
}

// double -> float rounded to nearest, ties away from zero (round to nearest even differs on
// exact ties only); magnitudes below the smallest normal float give a signed zero, above the
// largest finite one inf; inf stays inf and nan stays nan.  The rounding carry runs into the exponent field.
__device__ __forceinline__ float d2f_round(double x) {
    const uint32_t uh = (uint32_t)__double2hiint(x), ul = (uint32_t)__double2loint(x);
    const uint32_t e = (uh >> 20) & 0x7ffu;
    uint32_t v = ((((uh << 3) | (ul >> 29)) - (896u << 23)) + ((ul >> 28) & 1u)) & 0x7fffffffu;
    v = e < 897u ? 0u : v;
    // exponent field 2047: a nan (non-zero fraction) stays a quiet nan, +-inf stays inf
    const uint32_t special = ((uh & 0xfffffu) | ul) ? 0x7fc00000u : 0x7f800000u;
    v = e > 1150u ? (e == 2047u ? special : 0x7f800000u) : v;
    return __uint_as_float(v | (uh & 0x80000000u));
}

// x = hi + lo (double-float): hi = x rounded to float, lo = the rest (exact in double) rounded;
// one fp64 subtraction
__device__ __forceinline__ float2 d2df(double x) {
    const float h = d2f_round(x);
    return make_float2(h, d2f_round(x - f2d_exact(h)));
}

// hi + lo as a double: one fp64 addition
__device__ __forceinline__ double df2d(float hi, float lo) { return f2d_exact(hi) + f2d_exact(lo); }

}  // namespace usfft
