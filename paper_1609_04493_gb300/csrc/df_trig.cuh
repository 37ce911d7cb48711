// df_trig.cuh -- sine and cosine of an FP64 angle as double-float values
// (df.cuh), for the double-float kernels of FP64 data.
//
// Reduction (Cody and Waite): k = nearest integer to x (2 / pi) and
// r = x - k pi/2 with pi/2 split into two doubles, in two FP64 fused
// multiply-adds; |r| <= pi/4 up to rounding. The head of the split is the
// double nearest pi/2 and the tail the double nearest the remainder, so
// head + tail is pi/2 to 1.5e-33.
//
// Then the Taylor series of sin r and cos r about 0, whose coefficients are
// the inverse factorials. For |r| <= 0.8 the first omitted terms (r^17 / 17!
// for the sine, r^18 / 18! for the cosine) are below 1e-16. Terms below 3e-9
// of the result (r^11 on for the sine, r^12 on for the cosine) are summed in
// FP32, where the coefficients' own rounding costs about 2e-16; the rest run
// in double-float arithmetic. The quadrant k mod 4 then permutes and negates
// (sin r, cos r).
#pragma once
#include "df.cuh"

namespace rdyn {

constexpr double kDfTwoOverPi = 0.63661977236758134;   // 2 / pi
constexpr double kDfPio2Head = 1.5707963267948966;     // pi / 2, nearest double
constexpr double kDfPio2Tail = 6.123233995736766e-17;  // pi / 2 - head, nearest double

__device__ __forceinline__ void df_sincos(double x, DF *s_out, DF *c_out)
{
    const double k = rint(x * kDfTwoOverPi);
    const double rd = fma(-k, kDfPio2Tail, fma(-k, kDfPio2Head, x));
    const DF r = df_from_double(rd);
    const DF r2 = r * r;
    const float r2f = r2.hi;

    // sin r = r + r^3 (-1/3! + r^2/5! - ...)
    constexpr DF s3 = df_split_host(-1.0 / 6.0);
    constexpr DF s5 = df_split_host(1.0 / 120.0);
    constexpr DF s7 = df_split_host(-1.0 / 5040.0);
    constexpr DF s9 = df_split_host(1.0 / 362880.0);
    constexpr float s11 = (float)(-1.0 / 39916800.0);
    constexpr float s13 = (float)(1.0 / 6227020800.0);
    constexpr float s15 = (float)(-1.0 / 1307674368000.0);
    DF ps = DF(fmaf(fmaf(s15, r2f, s13), r2f, s11));
    ps = fma(ps, r2, s9);
    ps = fma(ps, r2, s7);
    ps = fma(ps, r2, s5);
    ps = fma(ps, r2, s3);
    const DF sr = fma(r * r2, ps, r);

    // cos r = 1 + r^2 (-1/2! + r^2/4! - ...)
    constexpr DF c4 = df_split_host(1.0 / 24.0);
    constexpr DF c6 = df_split_host(-1.0 / 720.0);
    constexpr DF c8 = df_split_host(1.0 / 40320.0);
    constexpr DF c10 = df_split_host(-1.0 / 3628800.0);
    constexpr float c12 = (float)(1.0 / 479001600.0);
    constexpr float c14 = (float)(-1.0 / 87178291200.0);
    constexpr float c16 = (float)(1.0 / 20922789888000.0);
    DF pc = DF(fmaf(fmaf(c16, r2f, c14), r2f, c12));
    pc = fma(pc, r2, c10);
    pc = fma(pc, r2, c8);
    pc = fma(pc, r2, c6);
    pc = fma(pc, r2, c4);
    pc = fma(pc, r2, DF(-0.5f));
    const DF cr = fma(pc, r2, DF(1.0f));

    // x = k pi/2 + r: quadrant k mod 4 (two's complement covers k < 0)
    const int qk = (int)k;
    DF sv = (qk & 1) ? cr : sr;
    DF cv = (qk & 1) ? sr : cr;
    if (qk & 2) sv = -sv;
    if ((qk + 1) & 2) cv = -cv;
    *s_out = sv;
    *c_out = cv;
}

}  // namespace rdyn
