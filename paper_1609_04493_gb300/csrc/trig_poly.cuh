// trig_poly.cuh -- FP32 sine and cosine of a joint angle on the FMA pipe.
//
// Method: Cody and Waite's additive range reduction (W. J. Cody, W. Waite,
// "Software Manual for the Elementary Functions", 1980): k = nearest integer
// to x * 2/pi, r = x - k * pi/2 with pi/2 split into three floats so that
// r is accurate to well below an ulp, |r| <= pi/4. Then
//     sin r = r + r^3 P(r^2),   cos r = 1 + r^2 Q(r^2),
// with P of degree 2 and Q of degree 3 whose constant term is -1/2, fitted by
// Lawson's iteratively reweighted least squares (minimax) on 400 Chebyshev nodes
// of [0, pi/4]: sin for relative error, cos - 1 + r^2/2 for absolute error.
// With the coefficients rounded to FP32 the polynomials are within 9e-9
// (relative, sin) and 6e-10 (absolute, cos) of the functions in exact
// arithmetic. tests/test_trig_fit_cpu.py repeats the fit and checks both.
// The quadrant k mod 4 selects and signs the pair. The integer k comes from the float rounding trick: adding
// 1.5 * 2^23 leaves k in the low mantissa bits.
//
// Absolute error about 7e-8 (under one ulp of 1.0) for |x| <= 1e5; no branch,
// no table, no special-function unit. Beyond |x| ~ 4e6 the reduction no longer
// holds (joint angles in radians are far below that).
#pragma once
#include <cuda_runtime.h>

namespace rdyn {

__device__ __forceinline__ void sincos_poly(float x, float *s, float *c)
{
    const float kMagic = 12582912.0f;  // 1.5 * 2^23
    const float t = fmaf(x, 6.3661975e-01f, kMagic);
    const float k = t - kMagic;
    const int quad = __float_as_int(t);
    float r = fmaf(-k, 1.5707964e+00f, x);
    r = fmaf(-k, -4.371139e-08f, r);
    r = fmaf(-k, -1.7763568e-15f, r);
    const float r2 = r * r;
    const float ps = fmaf(fmaf(-1.9515281e-04f, r2, 8.33216e-03f), r2, -1.6666655e-01f);
    const float sr = fmaf(r * r2, ps, r);
    const float pc = fmaf(fmaf(fmaf(2.44384519e-05f, r2, -1.38873677e-03f), r2, 4.16666456e-02f),
                          r2, -0.5f);
    const float cr = fmaf(r2, pc, 1.0f);
    const bool swap = (quad & 1) != 0;
    const float a = swap ? cr : sr;
    const float b = swap ? sr : cr;
    *s = __int_as_float(__float_as_int(a) ^ ((quad & 2) << 30));
    *c = __int_as_float(__float_as_int(b) ^ (((quad + 1) & 2) << 30));
}

}  // namespace rdyn
