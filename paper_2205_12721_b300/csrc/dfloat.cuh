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

#include <type_traits>

namespace tmop {

// Bit-level conversions between double and float pairs that use only the
// integer and FP32 pipes (B300's FP64 pipe, which also executes the F2F
// conversions to and from double, is the scarce resource).  Values outside
// the range where both words are normal floats take the plain conversion.
__host__ __device__ __forceinline__ unsigned long long dbits(double v)
{
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(v);
#else
    unsigned long long b;
    __builtin_memcpy(&b, &v, 8);
    return b;
#endif
}
__host__ __device__ __forceinline__ double from_dbits(unsigned long long b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double v;
    __builtin_memcpy(&v, &b, 8);
    return v;
#endif
}
__host__ __device__ __forceinline__ unsigned fbits(float v)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(v);
#else
    unsigned b;
    __builtin_memcpy(&b, &v, 4);
    return b;
#endif
}
__host__ __device__ __forceinline__ float from_fbits(unsigned b)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float v;
    __builtin_memcpy(&v, &b, 4);
    return v;
#endif
}

// float -> double by assembling the bits (exact for normal floats and zero)
__host__ __device__ __forceinline__ double f2d_bits(float f)
{
    const unsigned b = fbits(f);
    const unsigned e = (b >> 23) & 0xFFu;
    if (e == 0u || e == 0xFFu) return (double)f;            // zero, subnormal, inf, nan
    const unsigned long long s = (unsigned long long)(b >> 31) << 63;
    return from_dbits(s | ((unsigned long long)(e - 127u + 1023u) << 52) |
                      ((unsigned long long)(b & 0x7FFFFFu) << 29));
}

struct df {
    float h, l;
    df() = default;
    __host__ __device__ __forceinline__ df(float hi, float lo) : h(hi), l(lo) {}
    // h = rn(v), l = rn(v - h): conversions on the FP64 pipe
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

// The same split built from the bits on the integer/FP32 pipes, for kernels
// whose FP64 pipe is the bottleneck: h = v rounded to 24 significant bits,
// l = the signed remainder (29 bits rounded to 24), |l| <= ulp(h)/2.
__host__ __device__ __forceinline__ df df_bits(double v)
{
    const unsigned long long b = dbits(v);
    const int e = (int)((b >> 52) & 0x7FF);
    const int fe = e - 1023 + 127;                      // float exponent of h
    const int se = e - 1075 + 127;                      // float exponent of 2^(e-1075)
    if (fe <= 0 || fe >= 254 || se <= 0) return df(v);
    const unsigned sign = (unsigned)(b >> 63) << 31;
    unsigned hb = sign | ((unsigned)fe << 23) | (unsigned)((b >> 29) & 0x7FFFFFull);
    int r = (int)(b & 0x1FFFFFFFull);                   // dropped 29 fraction bits
    if (r >= (1 << 28)) {                               // round the magnitude up
        hb += 1u;
        r -= (1 << 29);
    }
    const float lv = (float)r * from_fbits((unsigned)se << 23);
    return df(from_fbits(hb), sign ? -lv : lv);
}

// double from a float pair on the integer pipe plus one FP64 add.
__host__ __device__ __forceinline__ double d_bits(const df &x) { return f2d_bits(x.h) + f2d_bits(x.l); }

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

// The high product is __fmul_rn: a plain multiply may be contracted by the
// compiler into an FMA with the TwoSum addition that consumes it, which
// breaks the exactness of the error-free transformation (observed: errors
// of ~1e-8 relative in the gradient of the I2 metrics).
__device__ __forceinline__ dprod operator*(const df &a, const df &b)
{
    const float p = __fmul_rn(a.h, b.h);
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

__device__ __forceinline__ df operator-(const df &a) { return df(-a.h, -a.l); }
__device__ __forceinline__ dprod operator-(const dprod &a) { return {-a.p, -a.e}; }
// a*b - c*d, normalised
__device__ __forceinline__ df dw_fms(const df &a, const df &b, const df &c, const df &d)
{
    const dprod p = a * b, r = c * d;
    return add_norm(p.p, -r.p, p.e - r.e);
}

// 2 x, exact
__device__ __forceinline__ df twice(const df &a) { return df(2.0f * a.h, 2.0f * a.l); }
__device__ __forceinline__ float twice(float a) { return 2.0f * a; }
__device__ __forceinline__ double twice(double a) { return 2.0 * a; }

// A normalised double-float value stored as the type of the stored data.
template <class RH> __device__ __forceinline__ RH store_dw(const df &a);
template <> __device__ __forceinline__ df store_dw<df>(const df &a) { return a; }
template <> __device__ __forceinline__ float store_dw<float>(const df &a) { return a.h; }

// Normalised value of a product.
__device__ __forceinline__ df to_df(const dprod &a) { return fast_two_sum(a.p, a.e); }
__device__ __forceinline__ df to_df(const df &a) { return a; }

// Assembly sums.  Float element vectors are summed on the FP32 pipes in a
// float-pair accumulator (TwoSum of the high words, low words and rounding
// errors collected in the low word, renormalised every 8 entries): B300
// issues FP64 adds and float-to-double conversions ~60x slower than FP32
// ops, and the plain double sum of float entries was bound by them.  Double
// entries are summed in double (splitting them on the integer pipe cost
// more than it saved).
template <class RI> struct AsmAcc { using T = double; };
template <> struct AsmAcc<float> { using T = df; };
__device__ __forceinline__ void asm_zero(double &a) { a = 0.0; }
__device__ __forceinline__ void asm_zero(df &a) { a = df(0.0f, 0.0f); }
__device__ __forceinline__ void asm_add(double &a, double v) { a += v; }
__device__ __forceinline__ void asm_add(df &a, float v) { acc_add(a, dprod{v, 0.0f}); }
__device__ __forceinline__ void asm_renorm(double &) {}
__device__ __forceinline__ void asm_renorm(df &a) { a = norm(a); }
template <class RO> __device__ __forceinline__ RO asm_out(double a) { return RO(a); }
template <class RO> __device__ __forceinline__ RO asm_out(const df &a) { return RO(norm(a).h); }

// Element vectors of the double-float Hessian action: each entry is the
// (unnormalised) float pair of the element sum, stored in the 8 bytes of a
// double slot.  The action kernels then run no FP64-unit conversion on their
// output; the assembly sums the pairs in double-float (TwoSum of the high
// words, low words and rounding errors in the low word, renormalised every 8
// entries) and rounds once per DOF to double.
template <class RV, class RC> struct EvPair { static constexpr bool value = false; };
template <> struct EvPair<double, df> { static constexpr bool value = true; };
template <> struct AsmAcc<df> { using T = df; };
__device__ __forceinline__ void asm_add(df &a, const df &v) { acc_add(a, dprod{v.h, v.l}); }
template <> __device__ __forceinline__ double asm_out<double>(const df &a)
{
    return (double)a.h + (double)a.l;
}
// entry loads of the assembly (read-only path; float pairs as one 8-byte load)
__device__ __forceinline__ double ld_entry(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ld_entry(const float *p) { return __ldg(p); }
__device__ __forceinline__ df ld_entry(const df *p)
{
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return df(v.x, v.y);
}
__device__ __forceinline__ double ld_plain(const double *p) { return *p; }
__device__ __forceinline__ float ld_plain(const float *p) { return *p; }
__device__ __forceinline__ df ld_plain(const df *p)
{
    const float2 v = *reinterpret_cast<const float2 *>(p);
    return df(v.x, v.y);
}



// Conversions used by the templated kernels.
__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ double to_d(const df &v) { return (double)v; }
// ... and the bit-level variants for FP64-pipe-bound kernels
__device__ __forceinline__ double to_db(double v) { return v; }
__device__ __forceinline__ double to_db(float v) { return f2d_bits(v); }
__device__ __forceinline__ double to_db(const df &v) { return d_bits(v); }
template <class R> __device__ __forceinline__ R from_db(double v) { return R(v); }
template <> __device__ __forceinline__ df from_db<df>(double v) { return df_bits(v); }

template <class R>
__device__ __forceinline__ R from_d(double v) { return (R)v; }
template <>
__device__ __forceinline__ df from_d<df>(double v) { return df(v); }

// Store of an action element-vector entry: the float pair (EvPair) or the
// value rounded to RV.
template <class RV, class RC>
__device__ __forceinline__ void ev_store(RV *p, const RC &a)
{
    if constexpr (EvPair<RV, RC>::value)
        *reinterpret_cast<float2 *>(p) = make_float2(a.h, a.l);
    else if constexpr (std::is_same<RV, RC>::value)
        *p = a;
    else
        *p = RV(to_d(a));
}
// *p += a on an action element-vector entry (terms added after the main
// action kernel, before the assembly).
template <class RV, class RC>
__device__ __forceinline__ void ev_accum(RV *p, const RC &a)
{
    if constexpr (EvPair<RV, RC>::value) {
        const float2 o = *reinterpret_cast<const float2 *>(p);
        const df s = df(o.x, o.y) + a;
        *reinterpret_cast<float2 *>(p) = make_float2(s.h, s.l);
    } else {
        *p = RV(to_d(*p) + to_d(a));
    }
}

// Per-DOF arithmetic of the MINRES vector kernels in the type S of the
// vectors' updates: double for FP64 vectors; float for FP32 vectors (the
// vectors are FP32 already; the float <-> double conversions and FP64 adds of
// a double evaluation ran on B300's FP64 pipe and bounded these kernels).
template <class R> using VecS = typename std::conditional<std::is_same<R, float>::value, float, double>::type;

// Dot-product partial sums: double for FP64 vectors; for FP32 vectors the
// exact float products summed in double-float on the FP32 pipes (TwoProd and
// TwoSum), converted to double once per thread.
template <class R> struct VecDot {
    double s = 0.0;
    __device__ __forceinline__ void add(R a, R b) { s += (double)a * (double)b; }
    __device__ __forceinline__ double get() const { return s; }
};
template <> struct VecDot<float> {
    df s = df(0.0f, 0.0f);
    __device__ __forceinline__ void add(float a, float b)
    {
        const float p = __fmul_rn(a, b);
        acc_add(s, dprod{p, fmaf(a, b, -p)});
    }
    __device__ __forceinline__ double get() const { return (double)s.h + (double)s.l; }
};

}  // namespace tmop
