// kg_arith.cuh -- scalar and complex arithmetic for the three FFT precisions.
//
//   double : IEEE FP64 (runs on the FP64 pipe, about 1/64 of the FP32 issue rate on GB300)
//   float  : IEEE FP32
//   df     : double-float, an unevaluated sum hi + lo of two floats (~48-bit significand),
//            built from Knuth's error-free two-sum (TAOCP vol. 2, 4.2.2) and Dekker's
//            exact product (Dekker 1971), here with the product error taken by one FMA.
//
// All float operations use the explicit round-to-nearest intrinsics so that the
// compiler cannot contract or reassociate the error-free transformations.
//
// Conversions between FP64 and the float formats are done with integer operations:
// on this GPU the cvt.f32.f64 / cvt.f64.f32 instructions share the slow FP64 pipe,
// while integer and FP32 instructions issue at the full rate.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace kg {

// ---------------------------------------------------------------------------
// double-float
// ---------------------------------------------------------------------------
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo) { df r; r.hi = hi; r.lo = lo; return r; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df_make(s, e);
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return df_make(s, e);
}

__device__ __forceinline__ df operator+(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ df operator-(df x) { return df_make(-x.hi, -x.lo); }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }

__device__ __forceinline__ df operator*(df x, df y) {
    float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

// sum without the final renormalisation: hi is the rounded sum of the high parts and lo
// collects the exact rounding error of that sum plus both low parts.  The pair still
// represents x + y to within u^2 (|x| + |y|), but |lo| may exceed half an ulp of hi, so a
// chain of such sums ends with df_norm.
__device__ __forceinline__ df df_add_lazy(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    return df_make(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ df df_sub_lazy(df x, df y) { return df_add_lazy(x, df_make(-y.hi, -y.lo)); }
__device__ __forceinline__ df df_norm(df x) { return fast_two_sum(x.hi, x.lo); }

// a.hi b.hi + c.hi d.hi + (low-order terms) without the final renormalisation: the two
// products are split exactly by FMA, their high parts added by two-sum, and every
// remaining term (product errors, cross terms with the low parts, the two-sum error)
// summed in float into the low part.  The pair represents the dot product to within
// u^2 (|ab| + |cd|) like df_add_lazy's results; inside a transform it only meets lazy
// sums and further products, and a transform's last stage renormalises.
__device__ __forceinline__ df df_dot2_lazy(df a, df b, df c, df d) {
    const float p1 = __fmul_rn(a.hi, b.hi);
    const float p2 = __fmul_rn(c.hi, d.hi);
    const df s = two_sum(p1, p2);
    float e = __fmaf_rn(a.hi, b.hi, -p1);           // exact error of p1
    e = __fadd_rn(e, __fmaf_rn(c.hi, d.hi, -p2));   // plus exact error of p2
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    e = __fmaf_rn(c.hi, d.lo, e);
    e = __fmaf_rn(c.lo, d.hi, e);
    return df_make(s.hi, __fadd_rn(s.lo, e));
}

// x y with the product's error taken by FMA and no final renormalisation (as df_dot2_lazy)
__device__ __forceinline__ df df_mul_lazy(df x, df y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return df_make(p, e);
}

// multiplication by a power of two (exact unless it under/overflows)
__device__ __forceinline__ df df_scale2(df x, float p2) { return df_make(__fmul_rn(x.hi, p2), __fmul_rn(x.lo, p2)); }
__device__ __forceinline__ float df_abs_hi(df x) { return fabsf(x.hi); }

// ---------------------------------------------------------------------------
// integer-only conversions
// ---------------------------------------------------------------------------
// float -> double, exact for normal floats; zero and subnormals give +-0; inf/nan kept.
__device__ __forceinline__ double f2d_int(float f) {
    uint32_t b = __float_as_uint(f);
    uint32_t sign = b & 0x80000000u, t = b & 0x7FFFFFFFu;
    uint32_t hw = ((t >> 3) + (896u << 20)) | sign;
    uint32_t lw = t << 29;
    if (t < 0x00800000u) { hw = sign; lw = 0u; }
    if (t >= 0x7F800000u) { hw = sign | 0x7FF00000u | (t > 0x7F800000u ? 0x00080000u : 0u); lw = 0u; }
    return __hiloint2double((int)hw, (int)lw);
}

// double -> float, round half away from zero on the magnitude; |d| < 2^-126 gives +-0,
// beyond the float range +-inf; nan stays nan.
__device__ __forceinline__ float d2f_int(double d) {
    uint32_t lw = (uint32_t)__double2loint(d), hw = (uint32_t)__double2hiint(d);
    uint32_t sign = hw & 0x80000000u, t = hw & 0x7FFFFFFFu;
    bool isnan_ = (t > 0x7FF00000u) || (t == 0x7FF00000u && lw != 0u);
    uint32_t lw2 = lw + 0x10000000u;
    uint32_t t2 = t + (lw2 < lw ? 1u : 0u);
    uint32_t fb = ((t2 - (896u << 20)) << 3) | (lw2 >> 29);
    uint32_t e = t2 >> 20;
    if (e < 897u) fb = 0u;
    if (e > 1150u) fb = 0x7F800000u;
    if (isnan_) fb = 0x7FC00000u;
    return __uint_as_float(fb | sign);
}

// double -> double-float: hi = d truncated to 24 significant bits, lo = the remaining
// 29 bits rounded to a float.  |d| < 2^-126 gives 0; beyond the float range inf (nan kept).
__device__ __forceinline__ df d2df_int(double d) {
    uint32_t lw = (uint32_t)__double2loint(d), hw = (uint32_t)__double2hiint(d);
    uint32_t sign = hw & 0x80000000u, t = hw & 0x7FFFFFFFu;
    uint32_t e = t >> 20;
    uint32_t hib = (((t - (896u << 20)) << 3) | (lw >> 29)) | sign;
    uint32_t r = lw & 0x1FFFFFFFu;
    float r1 = __fsub_rn(__uint_as_float(0x4B000000u | (r >> 6)), 8388608.0f);   // exact
    float r0 = __fsub_rn(__uint_as_float(0x4B000000u | (r & 63u)), 8388608.0f);  // exact
    float rf = __fmaf_rn(r1, 64.0f, r0);                                          // float(r)
    float lo = __fmul_rn(rf, __uint_as_float(((e - 948u) << 23) | sign));        // r 2^(e-1075)
    if (e < 949u) lo = 0.0f;
    if (e < 897u) hib = sign;
    if (e > 1150u) {
        bool isnan_ = (t > 0x7FF00000u) || (t == 0x7FF00000u && lw != 0u);
        hib = sign | (isnan_ ? 0x7FC00000u : 0x7F800000u);
        lo = 0.0f;
    }
    return df_make(__uint_as_float(hib), lo);
}

// ---------------------------------------------------------------------------
// complex numbers over a real type R
// ---------------------------------------------------------------------------
template <class R>
struct cx {
    R re, im;
};

template <class R>
__device__ __forceinline__ cx<R> cmake(R re, R im) { cx<R> c; c.re = re; c.im = im; return c; }
template <class R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return cmake<R>(a.re + b.re, a.im + b.im); }
template <class R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return cmake<R>(a.re - b.re, a.im - b.im); }
template <class R>
__device__ __forceinline__ cx<R> conj(cx<R> a) { return cmake<R>(a.re, -a.im); }
template <class R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
    return cmake<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// a * (S i), S = +-1
template <int S, class R>
__device__ __forceinline__ cx<R> mul_si(cx<R> a) {
    return S > 0 ? cmake<R>(-a.im, a.re) : cmake<R>(a.im, -a.re);
}
// a * i
template <class R>
__device__ __forceinline__ cx<R> mul_i(cx<R> a) { return cmake<R>(-a.im, a.re); }

// ---------------------------------------------------------------------------
// precision traits: storage of one complex value in HBM / shared memory,
// conversion from an FP64 value, and the real constants the butterflies need
// ---------------------------------------------------------------------------
struct PrecF64 {
    typedef double R;
    typedef double2 S;  // (re, im)
    static constexpr int kStoreBytes = 16;
    static __device__ __forceinline__ cx<R> load(const S& s) { return cmake<R>(s.x, s.y); }
    static __device__ __forceinline__ S pack(cx<R> c) { return make_double2(c.re, c.im); }
    static __device__ __forceinline__ R from_f64(double d) { return d; }
    static __device__ __forceinline__ R from_f32(float f) { return (double)f; }
    static __device__ __forceinline__ R rsqrt2() { return 0.70710678118654752440; }
    static __device__ __forceinline__ R scale2(R x, double p2) { return x * p2; }
    // acc + s * x with x in this precision, everything else FP64
    static __device__ __forceinline__ double fma_into(double s, R x, double acc) { return fma(s, x, acc); }
    // butterfly arithmetic: sums that may leave the pair unnormalised (double-float only),
    // the normalisation that ends such a chain, and the twiddle product
    static __device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) { return a + b; }
    static __device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) { return a - b; }
    static __device__ __forceinline__ R radd(R a, R b) { return a + b; }
    static __device__ __forceinline__ R rsub(R a, R b) { return a - b; }
    static __device__ __forceinline__ cx<R> cnorm(cx<R> a) { return a; }
    static __device__ __forceinline__ cx<R> ctw(cx<R> a, cx<R> w) { return cmul(a, w); }
    static __device__ __forceinline__ R rmul(R a, R c) { return a * c; }
    static __device__ __forceinline__ R cube(R x, R lam) { return lam * (x * x * x); }
    // x with its sign bit xor-ed with m (m = 0 or 0x80000000): exact negation on demand
    static __device__ __forceinline__ R flip(R x, unsigned m) {
        return __hiloint2double(__double2hiint(x) ^ (int)m, __double2loint(x));
    }
};

struct PrecF32 {
    typedef float R;
    typedef float2 S;
    static constexpr int kStoreBytes = 8;
    static __device__ __forceinline__ cx<R> load(const S& s) { return cmake<R>(s.x, s.y); }
    static __device__ __forceinline__ S pack(cx<R> c) { return make_float2(c.re, c.im); }
    static __device__ __forceinline__ R from_f64(double d) { return d2f_int(d); }
    static __device__ __forceinline__ R rsqrt2() { return 0.70710678118654752440f; }
    static __device__ __forceinline__ R scale2(R x, double p2) { return x * (float)p2; }
    static __device__ __forceinline__ double fma_into(double s, R x, double acc) { return fma(s, f2d_int(x), acc); }
    static __device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) { return a + b; }
    static __device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) { return a - b; }
    static __device__ __forceinline__ R radd(R a, R b) { return a + b; }
    static __device__ __forceinline__ R rsub(R a, R b) { return a - b; }
    static __device__ __forceinline__ cx<R> cnorm(cx<R> a) { return a; }
    static __device__ __forceinline__ cx<R> ctw(cx<R> a, cx<R> w) { return cmul(a, w); }
    static __device__ __forceinline__ R rmul(R a, R c) { return a * c; }
    static __device__ __forceinline__ R cube(R x, R lam) { return lam * (x * x * x); }
    static __device__ __forceinline__ R flip(R x, unsigned m) { return __uint_as_float(__float_as_uint(x) ^ m); }
};

struct PrecDF {
    typedef df R;
    typedef float4 S;  // (re.hi, re.lo, im.hi, im.lo)
    static constexpr int kStoreBytes = 16;
    static __device__ __forceinline__ cx<R> load(const S& s) { return cmake<R>(df_make(s.x, s.y), df_make(s.z, s.w)); }
    static __device__ __forceinline__ S pack(cx<R> c) { return make_float4(c.re.hi, c.re.lo, c.im.hi, c.im.lo); }
    static __device__ __forceinline__ R from_f64(double d) { return d2df_int(d); }
    // sqrt(1/2) = 0.70710678118654752440 as hi + lo
    static __device__ __forceinline__ R rsqrt2() { return df_make(0x1.6a09e6p-1f, 0x1.9fcef4p-27f); }
    static __device__ __forceinline__ R scale2(R x, double p2) { return df_scale2(x, (float)p2); }
    static __device__ __forceinline__ double fma_into(double s, R x, double acc) {
        return fma(s, f2d_int(x.hi), fma(s, f2d_int(x.lo), acc));
    }
    static __device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) {
        return cmake<R>(df_add_lazy(a.re, b.re), df_add_lazy(a.im, b.im));
    }
    static __device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) {
        return cmake<R>(df_sub_lazy(a.re, b.re), df_sub_lazy(a.im, b.im));
    }
    static __device__ __forceinline__ R radd(R a, R b) { return df_add_lazy(a, b); }
    static __device__ __forceinline__ R rsub(R a, R b) { return df_sub_lazy(a, b); }
    static __device__ __forceinline__ cx<R> cnorm(cx<R> a) { return cmake<R>(df_norm(a.re), df_norm(a.im)); }
    // (a.re w.re - a.im w.im, a.re w.im + a.im w.re), left unnormalised (df_dot2_lazy):
    // inside a transform a twiddle product is followed by lazy sums or another product,
    // and the transform's last stage renormalises its outputs
    static __device__ __forceinline__ cx<R> ctw(cx<R> a, cx<R> w) {
        return cmake<R>(df_dot2_lazy(a.re, w.re, -a.im, w.im), df_dot2_lazy(a.re, w.im, a.im, w.re));
    }
    // a real constant times a (the sqrt(1/2) rotations of a radix-8 DFT), unnormalised
    static __device__ __forceinline__ R rmul(R a, R c) { return df_mul_lazy(a, c); }
    // lam x^3 of the x pass, unnormalised: it feeds the forward transform's lazy sums
    static __device__ __forceinline__ R cube(R x, R lam) {
        return df_mul_lazy(lam, df_mul_lazy(df_mul_lazy(x, x), x));
    }
    static __device__ __forceinline__ R flip(R x, unsigned m) {
        return df_make(__uint_as_float(__float_as_uint(x.hi) ^ m), __uint_as_float(__float_as_uint(x.lo) ^ m));
    }
};

}  // namespace kg
