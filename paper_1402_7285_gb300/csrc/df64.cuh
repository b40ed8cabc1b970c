// df: a real number as the unevaluated sum hi + lo of two FP32 values
// ("double-float"), about 48 significant bits, computed on the FP32 pipes.
//
// GB300 runs FP32 about 64x faster than FP64 (2 FP64 FMAs per clock per SM);
// the FP32 recurrence of the shifted COCG loses too much accuracy (its error
// grows with the iteration count), so the df precision mode keeps the panel
// vectors and the sparse products in df.  Building blocks (error-free
// transformations, Knuth / Dekker; FMA form of the product):
//   TwoSum(a, b):     s = a + b, e = (a - (s - bb)) + (b - bb), bb = s - a   (s + e = a + b exactly)
//   FastTwoSum(a, b): s = a + b, e = b - (s - a)            (|a| >= |b|)
//   TwoProd(a, b):    p = a b,   e = fma(a, b, -p)          (p + e = a b exactly)
// df add: TwoSum of the high parts, the low parts added to the error, then
// FastTwoSum renormalisation.  df multiply: TwoProd of the high parts plus the
// two cross products, then FastTwoSum.  df fma(a, b, c) = c + a b fuses both.
// Storage: 8 bytes per real (hi, lo), so a complex df is one float4.
#pragma once

#include "common.cuh"

struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ __forceinline__ df(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ __forceinline__ df(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __host__ __device__ __forceinline__ df(float v) : hi(v), lo(0.f) {}
    __host__ __device__ __forceinline__ df(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

// Rounded FP32 operations that the compiler may not contract into FMAs (an FMA
// would change the rounding the error-free transformations rely on).
#ifdef __CUDA_ARCH__
#define DF_ADD(a, b) __fadd_rn((a), (b))
#define DF_SUB(a, b) __fsub_rn((a), (b))
#define DF_MUL(a, b) __fmul_rn((a), (b))
#else
#define DF_ADD(a, b) ((a) + (b))
#define DF_SUB(a, b) ((a) - (b))
#define DF_MUL(a, b) ((a) * (b))
#endif

__host__ __device__ __forceinline__ df df_two_sum(float a, float b) {
    const float s = DF_ADD(a, b);
    const float bb = DF_SUB(s, a);
    return df(s, DF_ADD(DF_SUB(a, DF_SUB(s, bb)), DF_SUB(b, bb)));
}

__host__ __device__ __forceinline__ df df_fast_two_sum(float a, float b) {
    const float s = DF_ADD(a, b);
    return df(s, DF_SUB(b, DF_SUB(s, a)));
}

__host__ __device__ __forceinline__ df operator+(df x, df y) {
    const df s = df_two_sum(x.hi, y.hi);
    return df_fast_two_sum(s.hi, DF_ADD(s.lo, DF_ADD(x.lo, y.lo)));
}

__host__ __device__ __forceinline__ df operator-(df x) { return df(-x.hi, -x.lo); }
__host__ __device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }

__host__ __device__ __forceinline__ df operator*(df x, df y) {
    const float p = DF_MUL(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return df_fast_two_sum(p, e);
}

// c + a * b
__host__ __device__ __forceinline__ df fma(df a, df b, df c) {
    const float p = DF_MUL(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const df s = df_two_sum(c.hi, p);
    return df_fast_two_sum(s.hi, DF_ADD(s.lo, DF_ADD(e, c.lo)));
}

// Lazy accumulator of a sum of products a_k b_k: the high parts of the
// products are summed with TwoSum, everything below (product errors, cross
// terms, TwoSum errors) in one plain FP32 sum; a single renormalisation at the
// end.  12 FP32 operations per term instead of 15 for a normalised df fma.
struct DfSum {
    float s, c;
    __host__ __device__ __forceinline__ void zero() { s = c = 0.f; }
    __host__ __device__ __forceinline__ void add_prod(df a, df b) {
        const float p = DF_MUL(a.hi, b.hi);
        float e = fmaf(a.hi, b.hi, -p);
        e = fmaf(a.hi, b.lo, e);
        e = fmaf(a.lo, b.hi, e);
        const df t = df_two_sum(s, p);
        s = t.hi;
        c = DF_ADD(c, DF_ADD(t.lo, e));
    }
    // b exact in FP32 (no low part): 11 operations
    __host__ __device__ __forceinline__ void add_prod(df a, float b) {
        const float p = DF_MUL(a.hi, b);
        float e = fmaf(a.hi, b, -p);
        e = fmaf(a.lo, b, e);
        const df t = df_two_sum(s, p);
        s = t.hi;
        c = DF_ADD(c, DF_ADD(t.lo, e));
    }
    // a plain value (a product with 1): the same operations on s and c as
    // add_prod(1, x), without the multiplications
    __host__ __device__ __forceinline__ void add_val(df x) {
        const df t = df_two_sum(s, x.hi);
        s = t.hi;
        c = DF_ADD(c, DF_ADD(t.lo, x.lo));
    }
    __host__ __device__ __forceinline__ void add_val(float x) {
        const df t = df_two_sum(s, x);
        s = t.hi;
        c = DF_ADD(c, t.lo);
    }
    __host__ __device__ __forceinline__ df value() const { return df_fast_two_sum(s, c); }
};

// a * b and c + a * b for an FP32 operand b (its low part is zero); named, not
// overloaded, so that a double operand never binds to them by narrowing
__host__ __device__ __forceinline__ df mul_f(df a, float b) {
    const float p = DF_MUL(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return df_fast_two_sum(p, e);
}
__host__ __device__ __forceinline__ df fma_f(df a, float b, df c) {
    const float p = DF_MUL(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    const df s = df_two_sum(c.hi, p);
    return df_fast_two_sum(s.hi, DF_ADD(s.lo, DF_ADD(e, c.lo)));
}

__device__ __forceinline__ df ldg_val(const df *p) {
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return df(v.x, v.y);
}
__device__ __forceinline__ float ldg_val(const float *p) { return __ldg(p); }
__device__ __forceinline__ double ldg_val(const double *p) { return __ldg(p); }

__host__ __device__ __forceinline__ cpx<double> to64(cpx<df> a) { return mk((double)a.re, (double)a.im); }
