// fmm_fp64.cuh -- double-precision square root and division for the march and
// adjoint kernels, built to keep work off GB300's FP64 pipe.
//
// The FP64 pipe of GB300 runs double arithmetic and the float <-> double
// conversion instructions at the same low rate, so these helpers take
// single-precision seeds, move them between formats with integer operations
// on the IEEE 754 bit patterns (binary32 / binary64: exponent biases 127 /
// 1023, 23 / 52 fraction bits), and refine them with Newton steps in double.
// Operands outside [1e-30, 1e30] in magnitude (for a division: a divisor
// outside it, or a dividend above about 1e280, infinite or NaN) take the
// correctly rounded operation instead.
#pragma once

#include <cstdint>

namespace fmmgb {

// bit patterns of 1e-30 and 1e30 as binary64
constexpr long long kF64Lo = 0x39b4484bfeebc2a0ll;
constexpr long long kF64Hi = 0x46293e5939a08ceall;

// |v| in [1e-30, 1e30]: a positive normal value with a normal float image
__device__ __forceinline__ bool in_float_range(double v)
{
    const long long m = __double_as_longlong(v) & 0x7fffffffffffffffll;
    return m >= kF64Lo && m <= kF64Hi;
}

// double -> float, truncating the fraction: the exponent field is re-biased
// by 1023 - 127 = 896 and the top 23 fraction bits kept (sign preserved).
__device__ __forceinline__ float f32_of(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned mag = (hi & 0x7fffffffu) - (896u << 20);
    return __uint_as_float((hi & 0x80000000u) | (mag << 3) | (lo >> 29));
}

// float -> double, exact for normal floats (sign preserved).
__device__ __forceinline__ double f64_of(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned long long hi =
        (unsigned long long)((u & 0x80000000u) | (((u & 0x7fffffffu) >> 3) + (896u << 20)));
    return __longlong_as_double((long long)((hi << 32) | (unsigned long long)(u << 29)));
}

// sqrt(v), v >= 0: float estimates y of sqrt(v) and rh of 1/(2 sqrt(v))
// (relative errors eps <= 3.4e-7 and eta <= 3e-7: v truncated to a float,
// rsqrtf), one Newton step y + rh (v - y^2); relative error eps^2/2 +
// eta eps <= 1.6e-13 (measured worst over a log-uniform sweep: 3.4e-14).
__device__ __forceinline__ double sqrt_fp64(double v)
{
    const long long vb = __double_as_longlong(v);   // negative values sort below kF64Lo
    if (!(vb >= kF64Lo && vb <= kF64Hi))
        return sqrt(v);
    const float vf = f32_of(v);
    const float rf = rsqrtf(vf);
    const double y = f64_of(vf * rf);
    const double rh = f64_of(0.5f * rf);
    return fma(rh, fma(-y, y, v), y);
}

// a / b: a float reciprocal of b refined by two Newton steps (exact to
// double rounding), then one correction of the quotient; a few ulp.
__device__ __forceinline__ double div_fp64(double a, double b)
{
    // |a| at most 1e280 (bit pattern 0x7a0...): the Newton steps neither
    // overflow nor meet an infinite or NaN dividend
    if (!in_float_range(b) || (__double_as_longlong(a) & 0x7fffffffffffffffll) > 0x7a00000000000000ll)
        return a / b;
    double r = f64_of(1.0f / f32_of(b));
    r = r * fma(-b, r, 2.0);
    r = r * fma(-b, r, 2.0);
    const double q = a * r;
    return fma(r, fma(-q, b, a), q);
}

}  // namespace fmmgb
