// fmm_df.cuh -- the root of Algorithm 11 for double-precision grids, computed
// in double-float arithmetic (a value is an unevaluated sum hi + lo of two
// floats, about 46 significant bits) so that the FP64 pipe, which on GB300
// runs at 1/64 of the float rate, only does the four additions whose
// operands are of order psi: the two shifts delta_i = psi_i - m, the
// recombination of the root u, and t = m + u.  Everything of order h (the
// shifted values, the speed term, the discriminant, its square root and u)
// lives in the float pipe.
//
// Error-free transformations (Knuth's two-sum, Dekker's fast two-sum, the
// exact product a*b - fl(a*b) from one fused multiply-add) build the
// double-float sums and products; the square root takes a float estimate
// x * rsqrt(x) and one Newton step carried in double-float.
//
// Accuracy: for a causal root the discriminant is at least q/2 (q the speed
// term (h/F)^2), so no step cancels catastrophically and u carries a
// relative error of a few 1e-14, i.e. ~1e-16 absolute on a grid with
// h = 1/1024: far below the fp64 parity tolerance of 1e-12 max|psi| even
// summed along a path of a thousand cells.
#pragma once

#include "fmm_fp64.cuh"

namespace fmmgb {

struct dfl {
    float h, l;
};

__device__ __forceinline__ dfl df_fast_two_sum(float a, float b)
{
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ dfl df_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

// x + y (both of one sign, or a result not far below the operands)
__device__ __forceinline__ dfl df_add(dfl x, dfl y)
{
    const dfl s = df_two_sum(x.h, y.h);
    return df_fast_two_sum(s.h, s.l + (x.l + y.l));
}

__device__ __forceinline__ dfl df_neg(dfl x) { return {-x.h, -x.l}; }

// x * x
__device__ __forceinline__ dfl df_sqr(dfl x)
{
    const float p = x.h * x.h;
    const float e = fmaf(x.h, x.h, -p);
    return df_fast_two_sum(p, fmaf(2.0f * x.h, x.l, e));
}

// x * y
__device__ __forceinline__ dfl df_mul(dfl x, dfl y)
{
    const float p = x.h * y.h;
    const float e = fmaf(x.h, y.h, -p);
    return df_fast_two_sum(p, fmaf(x.h, y.l, fmaf(x.l, y.h, e)));
}

// k * x for a small integer k (exact product of the high part)
__device__ __forceinline__ dfl df_scale(dfl x, float k)
{
    const float p = k * x.h;
    const float e = fmaf(k, x.h, -p);
    return df_fast_two_sum(p, fmaf(k, x.l, e));
}

// sqrt(x), x.h > 0: float estimate and one Newton step in double-float
__device__ __forceinline__ dfl df_sqrt(dfl x)
{
    const float r = rsqrtf(x.h);
    const float s = x.h * r;
    const float res = fmaf(-s, s, x.h) + x.l;
    return df_fast_two_sum(s, res * (0.5f * r));
}

// x < y for normalized pairs (|l| at most half an ulp of h, as the
// operations above return them): then the high parts decide unless they are
// equal
__device__ __forceinline__ bool df_lt(dfl x, dfl y)
{
    return x.h < y.h || (x.h == y.h && x.l < y.l);
}

// A non-negative double of magnitude below 1e30 as a double-float: the value
// truncated to 24 significant bits (fmm_fp64.cuh's f32_of) plus the remaining
// fraction bits as a float (the low 29 bits of the double's fraction, of which
// the top 23 are kept), both built with integer operations.  The pair is not
// normalized (lo may reach a whole ulp of hi), so df_lt against it can order
// two values wrongly when they lie within a float ulp of each other.  Values below 2^-100 become 0 (an absolute error no Algorithm
// 11 operand of order h notices).
__device__ __forceinline__ dfl df_of(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned E = (unsigned)(b >> 52) & 0x7ffu;
    if (E < 923u)   // below 2^-100, or zero
        return {0.0f, 0.0f};
    const float hi = f32_of(v);
    // 2^(E-1046) * (1 + m/2^23) - 2^(E-1046) with m the fraction bits 6..28
    const unsigned ef = (E - 919u) << 23;
    const unsigned m = ((unsigned)b & 0x1fffffffu) >> 6;
    const float lo = __uint_as_float(ef | m) - __uint_as_float(ef);
    return {hi, lo};
}

// A double-float as a double (one double addition of the exactly converted
// parts; fmm_fp64.cuh's f64_of is exact for normal floats, and a zero part
// is mapped to zero).
__device__ __forceinline__ double df_to_double(dfl x)
{
    const double h = x.h == 0.0f ? 0.0 : f64_of(x.h);
    const double l = x.l == 0.0f ? 0.0 : f64_of(x.l);
    return h + l;
}

// Algorithm 11's root for sorted upwind values m <= v1 <= v2 (nd of them
// present: nd = 1 uses m only), speed term q = (h/F)^2 in [1e-30, 1e30].
// With delta_i = v_i - m the root is t = m + u, u the larger root of
// sum_i (u - delta_i)^2 = q over the set: u = (S + sqrt(k q - P)) / k with
// S = sum delta_i and P = sum_{i<j} (delta_i - delta_j)^2 (Lagrange's form of
// S^2 - k (Q - q), a sum of squares, so nothing cancels), causal when the
// largest delta is below u (kStrict: when the double root t = m + u exceeds
// the largest value); the largest value is dropped while the set is not
// causal.  Returns the number of values in the causal set (0: none, root
// +inf) and the root in t.
template <bool kStrict>
__device__ __forceinline__ int df_shifted_root(double m, double v1, double v2, int nd, double q,
                                               double &t)
{
    const double d1 = nd >= 2 ? v1 - m : 0.0;
    const double d2 = nd >= 3 ? v2 - m : 0.0;
    // operands far above the scale of q cannot be causal: clamp them into
    // the float range (an integer compare: both are >= 0)
    dfl D1 = df_of(__double_as_longlong(d1) < kF64Hi ? d1 : 1e30);
    dfl D2 = df_of(__double_as_longlong(d2) < kF64Hi ? d2 : 1e30);
    const dfl Q = df_of(q);
    const dfl third = {0.333333343267f, -9.93410748e-9f};   // 1/3 = hi + lo
#pragma unroll 1
    for (; nd != 0; --nd) {
        // S, P and k q over the current set (D2 = 0 once axis 2 is dropped,
        // D1 = 0 once axis 1 is)
        const dfl S = df_add(D1, D2);
        dfl P = df_sqr(D1);
        if (nd == 3)
            P = df_add(P, df_add(df_sqr(D2), df_sqr(df_add(D2, df_neg(D1)))));
        const dfl kq = df_scale(Q, (float)nd);
        const dfl disc = df_add(kq, df_neg(P));
        if (disc.h > 0.0f) {
            const dfl r = df_add(S, df_sqrt(disc));
            const dfl u = nd == 3 ? df_mul(r, third) : (nd == 2 ? dfl{0.5f * r.h, 0.5f * r.l} : r);
            if constexpr (kStrict) {
                // causal when the root exceeds the largest value of the set,
                // tested on the doubles the cell and its neighbours will hold
                // (the test on the shifted double-floats can pass by a
                // rounding step while t rounds to that value or below it; an
                // upwind set recorded for the adjoint must point strictly
                // downhill)
                const double tt = m + df_to_double(u);
                const double vmax = nd == 3 ? v2 : v1;
                if (nd == 1 || __double_as_longlong(vmax) < __double_as_longlong(tt)) {
                    t = tt;
                    return nd;
                }
            } else {
                // without a recorded set, the shifted test suffices: it can
                // err only where u and the largest delta lie within a float
                // ulp of each other, and there the two sets' roots agree to
                // about 1e-14 u
                const dfl dmax = nd == 3 ? D2 : D1;   // 0 when nd == 1
                if (df_lt(dmax, u)) {
                    t = m + df_to_double(u);
                    return nd;
                }
            }
        }
        if (nd == 3)
            D2 = {0.0f, 0.0f};
        else
            D1 = {0.0f, 0.0f};
    }
    return 0;
}

}  // namespace fmmgb
