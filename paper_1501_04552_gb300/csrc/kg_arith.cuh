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

// ---------------------------------------------------------------------------
// packed pairs.  Blackwell's FP32x2 instructions (add / sub / mul / fma .f32x2) apply one
// IEEE FP32 operation to both halves of a 64-bit register pair for the issue cost of one
// instruction; the FMA pipe does the same work per lane as for two scalar instructions,
// but the issue slots they free go to the integer, load/store and FP64 instructions of
// the same warp.  The double-float complex arithmetic of PrecDF keeps (re, im) of the
// high words in one pair and of the low words in another and runs, lane by lane, the same
// round-to-nearest operations as the scalar double-float forms above.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2swap(float2 a) { return make_float2(a.y, a.x); }

// a double-float complex value as two pairs: h = (re.hi, im.hi), l = (re.lo, im.lo)
struct dfc {
    float2 h, l;
};

// lazy sums (df_add_lazy / df_sub_lazy on both components)
__device__ __forceinline__ dfc dfc_add_lazy(dfc a, dfc b) {
    const float2 s = f2add(a.h, b.h), bb = f2sub(s, a.h);
    const float2 e = f2add(f2sub(a.h, f2sub(s, bb)), f2sub(b.h, bb));
    dfc r;
    r.h = s;
    r.l = f2add(e, f2add(a.l, b.l));
    return r;
}
__device__ __forceinline__ dfc dfc_sub_lazy(dfc a, dfc b) {
    const float2 s = f2sub(a.h, b.h), bb = f2sub(s, a.h);
    const float2 e = f2sub(f2sub(a.h, f2sub(s, bb)), f2add(b.h, bb));
    dfc r;
    r.h = s;
    r.l = f2add(e, f2sub(a.l, b.l));
    return r;
}
// renormalisation (fast two-sum on both components)
__device__ __forceinline__ dfc dfc_norm(dfc a) {
    const float2 s = f2add(a.h, a.l);
    dfc r;
    r.h = s;
    r.l = f2sub(a.l, f2sub(s, a.h));
    return r;
}
// a times the real double-float c in both components, unnormalised (df_mul_lazy)
__device__ __forceinline__ dfc dfc_rmul_lazy(dfc a, float2 ch, float2 cl) {
    const float2 p = f2mul(a.h, ch);
    float2 e = f2fma(a.h, ch, f2neg(p));
    e = f2fma(a.h, cl, e);
    e = f2fma(a.l, ch, e);
    dfc r;
    r.h = p;
    r.l = e;
    return r;
}
// lane-wise product of two pair values, unnormalised (df_mul_lazy per component)
__device__ __forceinline__ dfc dfc_mul_lazy(dfc a, dfc b) {
    const float2 p = f2mul(a.h, b.h);
    float2 e = f2fma(a.h, b.h, f2neg(p));
    e = f2fma(a.h, b.l, e);
    e = f2fma(a.l, b.h, e);
    dfc r;
    r.h = p;
    r.l = e;
    return r;
}
// twiddle w in pair form: rh = (w.re.hi, w.re.hi), ih = (-w.im.hi, w.im.hi), and the low words
struct dftw {
    float2 rh, ih, rl, il;
};
// a w, unnormalised: per lane the FMA-split dot product of df_dot2_lazy, on the pairs
// a = (a.re, a.im) times (w.re, w.re) plus (a.im, a.re) times (-w.im, w.im)
__device__ __forceinline__ dfc dfc_tw_lazy(dfc a, const dftw& w) {
    const float2 sh = f2swap(a.h), sl = f2swap(a.l);
    const float2 p1 = f2mul(a.h, w.rh), p2 = f2mul(sh, w.ih);
    const float2 s = f2add(p1, p2), bb = f2sub(s, p1);
    const float2 es = f2add(f2sub(p1, f2sub(s, bb)), f2sub(p2, bb));
    float2 e = f2fma(a.h, w.rh, f2neg(p1));          // exact error of p1
    e = f2add(e, f2fma(sh, w.ih, f2neg(p2)));        // plus exact error of p2
    e = f2fma(a.h, w.rl, e);
    e = f2fma(a.l, w.rh, e);
    e = f2fma(sh, w.il, e);
    e = f2fma(sl, w.ih, e);
    dfc r;
    r.h = s;
    r.l = f2add(es, e);
    return r;
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
    // a twiddle as ctw takes it: the table entry exp(-2 pi i j/N), conjugated for sg = +1
    typedef cx<R> TW;
    static __device__ __forceinline__ TW twl(const S& s, int sg) {
        return cmake<R>(s.x, flip(s.y, sg > 0 ? 0x80000000u : 0u));
    }
    // whole-value forms of the elementwise operations: a power-of-two scale, lam x^3 of each
    // component, a + i b, and -i a (exact)
    static __device__ __forceinline__ cx<R> cscale2(cx<R> a, double p2) { return cmake<R>(scale2(a.re, p2), scale2(a.im, p2)); }
    static __device__ __forceinline__ cx<R> ccube(cx<R> a, R lam) { return cmake<R>(cube(a.re, lam), cube(a.im, lam)); }
    static __device__ __forceinline__ cx<R> cadd_i(cx<R> a, cx<R> b) { return cmake<R>(rsub(a.re, b.im), radd(a.im, b.re)); }
    static __device__ __forceinline__ cx<R> cmul_negi(cx<R> a) { return cmake<R>(a.im, -a.re); }
    static constexpr bool kPacked = false;
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
    typedef cx<R> TW;
    static __device__ __forceinline__ TW twl(const S& s, int sg) {
        return cmake<R>(s.x, flip(s.y, sg > 0 ? 0x80000000u : 0u));
    }
    // whole-value forms of the elementwise operations: a power-of-two scale, lam x^3 of each
    // component, a + i b, and -i a (exact)
    static __device__ __forceinline__ cx<R> cscale2(cx<R> a, double p2) { return cmake<R>(scale2(a.re, p2), scale2(a.im, p2)); }
    static __device__ __forceinline__ cx<R> ccube(cx<R> a, R lam) { return cmake<R>(cube(a.re, lam), cube(a.im, lam)); }
    static __device__ __forceinline__ cx<R> cadd_i(cx<R> a, cx<R> b) { return cmake<R>(rsub(a.re, b.im), radd(a.im, b.re)); }
    static __device__ __forceinline__ cx<R> cmul_negi(cx<R> a) { return cmake<R>(a.im, -a.re); }
    static constexpr bool kPacked = false;
};

struct PrecDF {
    typedef df R;
    // (re.hi, im.hi, re.lo, im.lo): a 16-byte load leaves the high words and the low words
    // each in a register pair, the operands of the packed FP32x2 arithmetic
    typedef float4 S;
    static constexpr int kStoreBytes = 16;
    static __device__ __forceinline__ cx<R> load(const S& s) { return cmake<R>(df_make(s.x, s.z), df_make(s.y, s.w)); }
    static __device__ __forceinline__ S pack(cx<R> c) { return make_float4(c.re.hi, c.im.hi, c.re.lo, c.im.lo); }
    static __device__ __forceinline__ dfc split(cx<R> a) {
        dfc r;
        r.h = make_float2(a.re.hi, a.im.hi);
        r.l = make_float2(a.re.lo, a.im.lo);
        return r;
    }
    static __device__ __forceinline__ cx<R> join(dfc a) { return cmake<R>(df_make(a.h.x, a.l.x), df_make(a.h.y, a.l.y)); }
    static __device__ __forceinline__ R from_f64(double d) { return d2df_int(d); }
    // sqrt(1/2) = 0.70710678118654752440 as hi + lo
    static __device__ __forceinline__ R rsqrt2() { return df_make(0x1.6a09e6p-1f, 0x1.9fcef4p-27f); }
    static __device__ __forceinline__ R scale2(R x, double p2) { return df_scale2(x, (float)p2); }
    static __device__ __forceinline__ double fma_into(double s, R x, double acc) {
        return fma(s, f2d_int(x.hi), fma(s, f2d_int(x.lo), acc));
    }
    static __device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) { return join(dfc_add_lazy(split(a), split(b))); }
    static __device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) { return join(dfc_sub_lazy(split(a), split(b))); }
    static __device__ __forceinline__ R radd(R a, R b) { return df_add_lazy(a, b); }
    static __device__ __forceinline__ R rsub(R a, R b) { return df_sub_lazy(a, b); }
    static __device__ __forceinline__ cx<R> cnorm(cx<R> a) { return join(dfc_norm(split(a))); }
    // (a.re w.re - a.im w.im, a.re w.im + a.im w.re), left unnormalised (the FMA-split dot
    // product of df_dot2_lazy per component): inside a transform a twiddle product is
    // followed by lazy sums or another product, and a transform's last stage renormalises
    // a twiddle is the table entry (w.re.hi, w.im.hi, w.re.lo, w.im.lo) of exp(-2 pi i j/N),
    // conjugated for sg = +1; the product forms its pairs where it uses them
    typedef float4 TW;
    static __device__ __forceinline__ cx<R> ctw(cx<R> a, const TW& w) {
        dftw t;
        t.rh = make_float2(w.x, w.x);
        t.ih = make_float2(-w.y, w.y);
        t.rl = make_float2(w.z, w.z);
        t.il = make_float2(-w.w, w.w);
        return join(dfc_tw_lazy(split(a), t));
    }
    static __device__ __forceinline__ TW twl(const S& s, int sg) {
        const unsigned m = sg > 0 ? 0x80000000u : 0u;
        return make_float4(s.x, __uint_as_float(__float_as_uint(s.y) ^ m), s.z, __uint_as_float(__float_as_uint(s.w) ^ m));
    }
    // the elementwise operations on both components at once, lane by lane as the scalar
    // forms (df_scale2, cube, df_add_lazy); sign flips are products with +-1, exact.  The x
    // pass keeps its 1/N^3 scale and its cube scalar: with these packed forms there ptxas
    // spilled 432 bytes per thread at 64 registers (24 with the scalar ones)
    static __device__ __forceinline__ cx<R> cscale2(cx<R> a, double p2) {
        const float2 f = make_float2((float)p2, (float)p2);
        dfc x = split(a);
        x.h = f2mul(x.h, f);
        x.l = f2mul(x.l, f);
        return join(x);
    }
    static __device__ __forceinline__ cx<R> ccube(cx<R> a, R lam) {
        const dfc x = split(a);
        const dfc x2 = dfc_mul_lazy(x, x);
        const dfc x3 = dfc_mul_lazy(x2, x);
        dfc l;
        l.h = make_float2(lam.hi, lam.hi);
        l.l = make_float2(lam.lo, lam.lo);
        return join(dfc_mul_lazy(l, x3));
    }
    static __device__ __forceinline__ cx<R> cadd_i(cx<R> a, cx<R> b) {   // a + i b
        const float2 sg = make_float2(-1.0f, 1.0f);
        const dfc y = split(b);
        dfc ib;
        ib.h = f2mul(f2swap(y.h), sg);
        ib.l = f2mul(f2swap(y.l), sg);
        return join(dfc_add_lazy(split(a), ib));
    }
    static __device__ __forceinline__ cx<R> cmul_negi(cx<R> a) {          // -i a
        const float2 sg = make_float2(1.0f, -1.0f);
        const dfc y = split(a);
        dfc r;
        r.h = f2mul(f2swap(y.h), sg);
        r.l = f2mul(f2swap(y.l), sg);
        return join(r);
    }
    // x (1 + sg i)/sqrt2 and x (-1 + sg i)/sqrt2, the rotations of a radix-8 DFT
    static __device__ __forceinline__ cx<R> crot(cx<R> a, int sg, bool minus) {
        const float2 sgn = make_float2(-(float)sg, (float)sg);
        const dfc x = split(a);
        dfc y;                                   // (-sg x.im, sg x.re), exact
        y.h = f2mul(f2swap(x.h), sgn);
        y.l = f2mul(f2swap(x.l), sgn);
        const df r = rsqrt2();
        return join(dfc_rmul_lazy(minus ? dfc_sub_lazy(y, x) : dfc_add_lazy(x, y), make_float2(r.hi, r.hi),
                                  make_float2(r.lo, r.lo)));
    }
    static constexpr bool kPacked = true;
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
