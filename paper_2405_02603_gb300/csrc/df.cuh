// df.cuh -- double-float ("double-word") arithmetic: a value is hi + lo with
// two floats, |lo| <= ulp(hi)/2, about 48 significant bits.  On the GB300 the
// FP32 pipes are ~61x faster than FP64 (measured 73.9 vs 1.20 TFLOP/s), so the
// FP64-accuracy solve (FSP_F64_DF) runs its transforms in this arithmetic.
//
// Algorithms (error-free transformations, Knuth / Dekker; double-word
// operations as analysed by Joldes, Muller and Popescu, "Tight and rigorous
// error bounds for basic building blocks of double-word arithmetic", 2017):
//   two_sum(a,b):      s = a+b, v = s-a, e = (a-(s-v)) + (b-v)      (exact)
//   fast_two_sum(a,b): s = a+b, e = b-(s-a)            (exact if |a|>=|b|)
//   add:  "sloppy" double-word sum, error <= ~2^-47 (|x|+|y|) -- normwise
//         bounds are all an FFT needs
//   mul:  p = a.hi*b.hi, e = fma(a.hi,b.hi,-p) + a.hi*b.lo + a.lo*b.hi,
//         normalised with fast_two_sum
// Every operation uses the _rn intrinsics, which the compiler never fuses or
// reassociates: contracting a*b+c into an FMA would break the exactness of
// the transformations above.
#pragma once
#include <cuda_runtime.h>

namespace fsp {

struct df {
    float hi, lo;
    __host__ __device__ constexpr df() : hi(0.f), lo(0.f) {}
    // exact split of a double into the nearest float and the rounded rest
    __host__ __device__ constexpr df(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ constexpr df(float h, float l, int) : hi(h), lo(l) {}
    __host__ __device__ constexpr explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float v = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
    return df(s, e, 0);
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df(s, __fsub_rn(b, __fsub_rn(s, a)), 0);
}
__device__ __forceinline__ df operator+(df a, df b) {
    const df s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo, 0); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df &operator*=(df &a, df b) {
    a = a * b;
    return a;
}

struct __align__(16) cdf {
    df x, y;
};

template <typename T> struct cx;
template <> struct cx<df> { using t = cdf; };

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df df_from_double(double x) {
    const float h = __double2float_rn(x);
    return df(h, __double2float_rn(x - (double)h), 0);
}

// a*b + c*d for double-words, with one normalisation: the products' high parts
// are summed exactly (two_sum), their rounding errors and the cross terms are
// accumulated by FMAs into the low part.
__device__ __forceinline__ df df_dot2(df a, df b, df c, df d) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    const float q = __fmul_rn(c.hi, d.hi);
    const float f = __fmaf_rn(c.hi, d.hi, -q);
    const df s = df_two_sum(p, q);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    e = __fmaf_rn(c.hi, d.lo, e);
    e = __fmaf_rn(c.lo, d.hi, e);
    e = __fadd_rn(e, __fadd_rn(f, s.lo));
    return df_fast_two_sum(s.hi, e);
}

// complex multiply with one normalisation per component
__device__ __forceinline__ cdf cmul(cdf a, cdf b) {
    return cdf{df_dot2(a.x, b.x, -a.y, b.y), df_dot2(a.x, b.y, a.y, b.x)};
}

// read-only 16-byte load through the non-coherent path
__device__ __forceinline__ cdf ldg_c(const cdf *p) {
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    return cdf{df(q.x, q.y, 0), df(q.z, q.w, 0)};
}

}  // namespace fsp
