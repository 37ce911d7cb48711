// df.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi) / 2, a significand of about 48 bits.
//
// Methods: the exact sum a + b = s + e is Knuth's branch-free two-sum (TAOCP
// vol. 2, Sec. 4.2.2) and, for |a| >= |b|, Dekker's fast two-sum (T. J.
// Dekker, Numer. Math. 18, 1971); the exact product a b = p + e takes its
// error from one fused multiply-add. The sum of two double-floats adds the
// two low parts to the error of the high parts and renormalises once (the
// cheaper of Dekker's two additions): its error is a few units of 2^-48
// times |x| + |y|, the bound a double sum of inputs that carry rounding
// errors of their own already has. Products are accurate to a few units of
// 2^-48 of the result.
//
// On GB300 the FP32 pipe executes 64 times as many fused multiply-adds per
// clock as the FP64 pipe, so a double-float multiply-add (about 15 FP32
// instructions) costs a quarter of an FP64 one in issue time.
//
// The same helpers are overloaded for double, so code templated on the scalar
// D runs in either.
#pragma once
#include <cuda_runtime.h>

namespace rdyn {
// The type and its operators sit in a namespace of their own so that calls
// to fma inside rdyn find this overload by argument-dependent lookup only and
// do not hide the global fma(double, double, double).
namespace dfloat {

// 8-byte aligned, so a pair moves with one 64-bit load or store
struct alignas(8) DF {
    float hi, lo;
    DF() = default;
    __host__ __device__ constexpr DF(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr explicit DF(float h) : hi(h), lo(0.0f) {}
};

// exact a + b = s + e (Knuth)
__device__ __forceinline__ DF df_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return DF(s, (a - (s - bb)) + (b - bb));
}

// exact a + b = s + e for |a| >= |b| or a = 0 (Dekker)
__device__ __forceinline__ DF df_fast_two_sum(float a, float b)
{
    const float s = a + b;
    return DF(s, b - (s - a));
}

__device__ __forceinline__ DF operator+(DF x, DF y)
{
    const DF s = df_two_sum(x.hi, y.hi);
    return df_fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}

__device__ __forceinline__ DF operator-(DF x) { return DF(-x.hi, -x.lo); }
__device__ __forceinline__ DF operator-(DF x, DF y) { return x + (-y); }

__device__ __forceinline__ DF operator*(DF x, DF y)
{
    const float p = x.hi * y.hi;
    const float e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, fmaf(x.hi, y.hi, -p)));
    return df_fast_two_sum(p, e);
}

// x y + z: the product's exact high part and error terms, then one sum
__device__ __forceinline__ DF fma(DF x, DF y, DF z)
{
    const float p = x.hi * y.hi;
    const float e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, fmaf(x.hi, y.hi, -p)));
    const DF s = df_two_sum(p, z.hi);
    return df_fast_two_sum(s.hi, s.lo + (e + z.lo));
}

__device__ __forceinline__ DF &operator+=(DF &x, DF y) { return x = x + y; }
__device__ __forceinline__ DF &operator-=(DF &x, DF y) { return x = x - y; }

}  // namespace dfloat
using dfloat::DF;
using dfloat::df_two_sum;

// ---- helpers overloaded for double and DF

// x / 2 and 2 x (exact)
__device__ __forceinline__ double dhalf(double x) { return 0.5 * x; }
__device__ __forceinline__ DF dhalf(DF x) { return DF(0.5f * x.hi, 0.5f * x.lo); }
__device__ __forceinline__ double dtwice(double x) { return 2.0 * x; }
__device__ __forceinline__ DF dtwice(DF x) { return DF(2.0f * x.hi, 2.0f * x.lo); }
// 2 x + y: one FMA in double; the exact doubling and one sum in double-float
__device__ __forceinline__ double dtwice_add(double x, double y) { return fma(2.0, x, y); }
__device__ __forceinline__ DF dtwice_add(DF x, DF y) { return dtwice(x) + y; }

// 1 / x. DF: the FP32 reciprocal r refined by one Newton step
// r + r (1 - x r), which doubles its correct bits.
__device__ __forceinline__ double drecip(double x) { return 1.0 / x; }
__device__ __forceinline__ DF drecip(DF x)
{
    const float r = 1.0f / x.hi;
    const DF e = DF(1.0f) - x * DF(r);
    return fma(DF(r), e, DF(r));
}

__device__ __forceinline__ bool dpositive(double x) { return x > 0.0; }
__device__ __forceinline__ bool dpositive(DF x) { return x.hi > 0.0f; }
__device__ __forceinline__ bool disnan(double x) { return !(x == x); }
__device__ __forceinline__ bool disnan(DF x) { return !(x.hi == x.hi); }

// a - b of two data values in D: exact for FP32 data (a double, or a
// double-float, holds the difference of two floats exactly), one rounding for
// FP64 data
template <typename D>
struct DSub;
template <>
struct DSub<double> {
    __device__ __forceinline__ static double sub(float a, float b) { return (double)a - (double)b; }
    __device__ __forceinline__ static double sub(double a, double b) { return a - b; }
};
template <>
struct DSub<DF> {
    __device__ __forceinline__ static DF sub(float a, float b) { return df_two_sum(a, -b); }
};

template <typename D, typename T>
__device__ __forceinline__ D dsub_exact(T a, T b)
{
    return DSub<D>::sub(a, b);
}

// conversions between the data types (float, double) and D
template <typename To>
struct DCvt;
template <>
struct DCvt<double> {
    __device__ __forceinline__ static double from(float x) { return (double)x; }
    __device__ __forceinline__ static double from(double x) { return x; }
    __device__ __forceinline__ static double from(DF x) { return (double)x.hi + (double)x.lo; }
};
template <>
struct DCvt<float> {
    __device__ __forceinline__ static float from(float x) { return x; }
    __device__ __forceinline__ static float from(double x) { return (float)x; }
    __device__ __forceinline__ static float from(DF x) { return x.hi + x.lo; }
};
template <>
struct DCvt<DF> {
    __device__ __forceinline__ static DF from(float x) { return DF(x); }
    __device__ __forceinline__ static DF from(DF x) { return x; }
};

template <typename To, typename From>
__device__ __forceinline__ To dcvt(From x)
{
    return DCvt<To>::from(x);
}

// nearest double-float of a double (host side: records are split once;
// constexpr, so constant tables split at compile time)
constexpr DF df_split_host(double v)
{
    return DF((float)v, (float)(v - (double)(float)v));
}

// double <-> double-float on the device (conversions on the FP64 path)
__device__ __forceinline__ DF df_from_double(double v)
{
    const float hi = __double2float_rn(v);
    return DF(hi, __double2float_rn(v - (double)hi));
}

__device__ __forceinline__ double df_to_double(DF x) { return (double)x.hi + (double)x.lo; }

}  // namespace rdyn
