// Double-float ("double-word") arithmetic on the FP32 pipes.
//
// B300 issues FP32 FMAs ~60x faster than FP64 ones, so the FP64-accuracy
// contractions run on pairs of floats x = h + l (|l| <= ulp(h)/2, a 48-bit
// significand, unit roundoff ~2^-48 ~ 3.6e-15).  The building blocks are the
// classical error-free transformations: Knuth's TwoSum, Dekker's FastTwoSum
// and the FMA-based TwoProd (see Joldes, Muller, Popescu, "Tight and rigorous
// error bounds for basic building blocks of double-word arithmetic", ACM TOMS
// 2017).  Products keep the cross terms h*l and l*h; the l*l term is below
// the working precision.  Exponent range is FP32's (|x| in ~[1e-38, 3e38]).
#pragma once

#include <cuda_runtime.h>

namespace tmop {

struct df {
    float h, l;
    df() = default;
    __host__ __device__ __forceinline__ df(float hi, float lo) : h(hi), l(lo) {}
    // exact up to the 48-bit significand: h = rn(v), l = rn(v - h)
    __host__ __device__ __forceinline__ df(double v)
    {
        h = (float)v;
        l = (float)(v - (double)h);
    }
    __host__ __device__ __forceinline__ explicit operator double() const
    {
        return (double)h + (double)l;
    }
};

// An unnormalised product p + e (|e| small relative to |p|).
struct dprod {
    float p, e;
};

__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    const float s = a + b;
    return df(s, b - (s - a));
}

// (a + b) + lo, normalised: TwoSum of the high parts, low parts added to the
// rounding error, one FastTwoSum to renormalise.
__device__ __forceinline__ df add_norm(float a, float b, float lo)
{
    const float s = a + b;
    const float bb = s - a;
    float err = (a - (s - bb)) + (b - bb);
    err += lo;
    return fast_two_sum(s, err);
}

__device__ __forceinline__ dprod operator*(const df &a, const df &b)
{
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return {p, e};
}

__device__ __forceinline__ df &operator+=(df &a, const dprod &b)
{
    a = add_norm(a.h, b.p, a.l + b.e);
    return a;
}

__device__ __forceinline__ df &operator+=(df &a, const df &b)
{
    a = add_norm(a.h, b.h, a.l + b.l);
    return a;
}

__device__ __forceinline__ df operator+(const dprod &a, const dprod &b)
{
    return add_norm(a.p, b.p, a.e + b.e);
}

__device__ __forceinline__ df operator+(const df &a, const df &b)
{
    return add_norm(a.h, b.h, a.l + b.l);
}

// Unnormalised accumulation acc += a*b: exact TwoSum of the high parts, the
// low parts and the rounding error summed in the low word without the final
// renormalisation (|l| may grow to a few ulp(h) over a short sum; norm()
// restores the invariant).  Used for the fixed-length contractions.
__device__ __forceinline__ void acc_add(df &a, const dprod &b)
{
    const float s = a.h + b.p;
    const float bb = s - a.h;
    const float err = (a.h - (s - bb)) + (b.p - bb);
    a.l = a.l + b.e + err;
    a.h = s;
}
__device__ __forceinline__ void acc_add(double &a, double b) { a += b; }
__device__ __forceinline__ void acc_add(float &a, float b) { a += b; }

__device__ __forceinline__ df norm(const df &a) { return fast_two_sum(a.h, a.l); }
__device__ __forceinline__ double norm(double a) { return a; }
__device__ __forceinline__ float norm(float a) { return a; }

// Normalised value of a product.
__device__ __forceinline__ df to_df(const dprod &a) { return fast_two_sum(a.p, a.e); }
__device__ __forceinline__ df to_df(const df &a) { return a; }

// Conversions used by the templated kernels.
__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(const df &v) { return (double)v; }

template <class R>
__device__ __forceinline__ R from_d(double v) { return (R)v; }
template <>
__device__ __forceinline__ df from_d<df>(double v) { return df(v); }

}  // namespace tmop
