// kg_fft.cuh -- shared-memory Stockham FFTs and the pieces the passes of a step share.
//
// One time step of the scheme of section 1.1.2 (Eq. (2), stepped in Fourier space
// with the cube formed in real space, two 3D FFTs per step) is a sequence of passes
// over the work array W (half spectrum in x, [z][y][kx] / [kz][ky][kx], kx = 0..N/2
// fastest):
//
//   X  : per x-line, complex-to-real inverse along x, scale 1/N^3 -> u^n on the line;
//        max|u|, sum u^4; F = lam u^3; real-to-complex forward along x; in place.
//        (One line through an N/2-point complex FFT, or two lines through one N-point
//        complex FFT.)
//   Yf : per (z, kx) column, forward complex FFT along y, in place.
//   Z  : per (ky, kx) column, forward complex FFT along z -> F^n_k; per mode, the FP64
//        update uh^{n+1} = 2 c_k uh^n - uh^{n-1} + 2 beta_k F^n_k written over uh^{n-1},
//        optional Q^{n+1/2} partial sums; inverse complex FFT along z of uh^{n+1}, in
//        place (one kernel; the IEEE FP64 passes run the three parts as kernels Zf, U, Zi).
//   Yi : per (z, kx) column, inverse complex FFT along y, in place.
//
// The pencil transposes of a distributed 3D FFT become strided column accesses:
// a column tile is C consecutive kx columns (C * element = 128 bytes, one full
// line per row) by all N rows, held in registers (8 values per thread) and in
// shared memory between radix stages.
//
// FFT formulation: Stockham autosort, radix 8 (last stage radix 2 or 4 when log2 n
// is not a multiple of 3).  With T = n/8 threads per line, thread j holds the
// values of index j + T s (s = 0..7) before every stage and after the last one, so
// a forward transform can feed an inverse one without any exchange.
#pragma once
#include "kg_arith.cuh"

namespace kg {

// asynchronous 16-byte global -> shared copy (L2 only), and its completion wait
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// x-pass modes: one stepping pass, or a read-only pass for P^n
enum { MODE_STEP = 0, MODE_PEEK = 1 };

constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }

// Stage plan of a length-n transform: radix-8 stages and, when log2 n is not a multiple
// of 3, one radix-2 or radix-4 stage -- last (REMFIRST = false, the default) or first.
// Both orders compute the same DFT; the autotuner of the batched ensemble picks one.
template <int n, bool REMFIRST = false>
struct FftShape {
    static_assert(n >= 8 && (n & (n - 1)) == 0, "power-of-two length >= 8");
    static constexpr int lg = ilog2c(n);
    static constexpr int n8 = lg / 3;              // radix-8 stages
    static constexpr int rem = 1 << (lg % 3);      // radix of the short stage (1: none)
    static constexpr int stages = n8 + (rem > 1 ? 1 : 0);
    static constexpr int T = n / 8;                // threads per line
    static constexpr bool kRemFirst = REMFIRST && rem > 1;
    __host__ __device__ static constexpr int radix(int s) { return kRemFirst ? (s == 0 ? rem : 8) : (s < n8 ? 8 : rem); }
    __host__ __device__ static constexpr int span(int s) { return s == 0 ? 1 : span(s - 1) * radix(s - 1); }   // Ns of stage s
};

// The transform sign sg (-1 forward, +1 inverse) is an ordinary argument: where a call
// passes a literal the compiler folds every sign flip away, and a pass that runs both
// directions (the x and z passes) keeps one copy of the butterfly code for both.
__device__ __forceinline__ unsigned sign_mask(int sg) { return sg < 0 ? 0x80000000u : 0u; }

// twiddle exp(sg 2 pi i idx / Ntab) from a table of exp(-2 pi i j / Ntab); the table is
// in global memory (read through L1) or, in the FP32 column passes, a shared-memory copy
// (stage_table), so this is a plain load
template <class P>
__device__ __forceinline__ typename P::TW twiddle(const typename P::S* __restrict__ tw, int idx, int sg) {
    return P::twl(tw[idx], sg);   // conjugated for sg = +1
}

// w[s] = exp(sg 2 pi i (j + T s) / Ntab), s = 0..7, from two table loads and products
// (chains of at most four products): for passes bound by the L1TEX pipe
template <class P>
__device__ __forceinline__ void twiddle_run(const typename P::S* __restrict__ tw, int j, int T, int sg,
                                            cx<typename P::R> (&w)[8]) {
    typedef cx<typename P::R> C;
    const C wj = twiddle<P>(tw, j, sg), wt = twiddle<P>(tw, T, sg);
    const C t2 = cmul(wt, wt), t3 = cmul(t2, wt), t4 = cmul(t2, t2);
    const C t5 = cmul(t4, wt), t6 = cmul(t4, t2), t7 = cmul(t4, t3);
    w[0] = wj;
    w[1] = cmul(wj, wt);
    w[2] = cmul(wj, t2);
    w[3] = cmul(wj, t3);
    w[4] = cmul(wj, t4);
    w[5] = cmul(wj, t5);
    w[6] = cmul(wj, t6);
    w[7] = cmul(wj, t7);
}

// a * (sg i) = (-sg a.im, sg a.re)
template <class P>
__device__ __forceinline__ cx<typename P::R> mul_sgi(cx<typename P::R> a, int sg) {
    return cmake<typename P::R>(P::flip(a.im, sign_mask(-sg)), P::flip(a.re, sign_mask(sg)));
}

// ---------------------------------------------------------------------------
// small DFTs, y_k = sum_j u_j exp(sg 2 pi i j k / R), in place, natural order
// ---------------------------------------------------------------------------
// The sums inside one small DFT use P::cadd / P::csub, which for double-float skip the
// renormalisation; dft() renormalises the R outputs once at the end.
template <class P>
__device__ __forceinline__ void dft2(cx<typename P::R>* u) {
    cx<typename P::R> a = P::cadd(u[0], u[1]), b = P::csub(u[0], u[1]);
    u[0] = a;
    u[1] = b;
}

template <class P>
__device__ __forceinline__ void dft4(cx<typename P::R>* u, int sg) {
    typedef cx<typename P::R> C;
    C t0 = P::cadd(u[0], u[2]), t1 = P::csub(u[0], u[2]), t2 = P::cadd(u[1], u[3]);
    C t3 = mul_sgi<P>(P::csub(u[1], u[3]), sg);
    u[0] = P::cadd(t0, t2);
    u[1] = P::cadd(t1, t3);
    u[2] = P::csub(t0, t2);
    u[3] = P::csub(t1, t3);
}

template <class P, bool PROT = true>
__device__ __forceinline__ void dft8(cx<typename P::R>* u, int sg) {
    typedef typename P::R R;
    typedef cx<R> C;
    C a[4], b[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        a[j] = P::cadd(u[j], u[j + 4]);
        b[j] = P::csub(u[j], u[j + 4]);
    }
    if constexpr (P::kPacked && PROT) {   // the same two rotations on (re, im) pairs
        b[1] = P::crot(b[1], sg, false);
        b[3] = P::crot(b[3], sg, true);
    } else {
        const R r = P::rsqrt2();
        const unsigned ms = sign_mask(sg), mns = sign_mask(-sg);
        {   // b1 *= exp(sg i pi/4) = (1 + sg i)/sqrt2:  (x.re - sg x.im, x.im + sg x.re) / sqrt2
            C x = b[1];
            b[1] = cmake<R>(P::rmul(P::radd(x.re, P::flip(x.im, mns)), r), P::rmul(P::radd(x.im, P::flip(x.re, ms)), r));
        }
        {   // b3 *= exp(sg 3 i pi/4) = (-1 + sg i)/sqrt2:  (-sg x.im - x.re, sg x.re - x.im) / sqrt2
            C x = b[3];
            b[3] = cmake<R>(P::rmul(P::rsub(P::flip(x.im, mns), x.re), r), P::rmul(P::rsub(P::flip(x.re, ms), x.im), r));
        }
    }
    b[2] = mul_sgi<P>(b[2], sg);
    dft4<P>(a, sg);
    dft4<P>(b, sg);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        u[2 * k] = a[k];
        u[2 * k + 1] = b[k];
    }
}

// NORM: renormalise the outputs.  Between stages it is skipped: every output but the
// first meets a twiddle product next, which renormalises, and an unnormalised pair
// still represents its value to within u^2 times the sum of the magnitudes that formed it
// PROT: the rotations of a radix-8 DFT on packed pairs (precisions that have them); the
// column passes measured faster with the scalar form (0.572 against 0.592 ms per 512^3 y pass,
// double-float), the x and z passes with the packed one (1.196 against 1.217 ms, 1.779 against
// 1.816 ms)
template <class P, int RADIX, bool NORM = true, bool PROT = true>
__device__ __forceinline__ void dft(cx<typename P::R>* u, int sg) {
    if (RADIX == 8) dft8<P, PROT>(u, sg);
    else if (RADIX == 4) dft4<P>(u, sg);
    else if (RADIX == 2) dft2<P>(u);
    if (NORM) {
#pragma unroll
        for (int r = 0; r < RADIX; r++) u[r] = P::cnorm(u[r]);
    }
}

// Copy a twiddle table of n entries into shared memory once per CTA (all threads call
// it) when the values are 8-byte FP32 pairs: the FP32 column passes are limited by the
// L1TEX pipe, where the twiddle loads outnumber the data loads.  The 16-byte passes keep
// the table in L1: their FFT exchanges already fill the shared-memory bandwidth.
template <class S>
__device__ __forceinline__ const S* stage_table(const S* __restrict__ g, S* sm, int n) {
    if constexpr (sizeof(S) != 8) {
        return g;
    } else {
        for (int i = threadIdx.x; i < n; i += blockDim.x) sm[i] = g[i];
        __syncthreads();
        return sm;
    }
}

// ---------------------------------------------------------------------------
// shared-memory views
// ---------------------------------------------------------------------------
// column tile: element (row, column c) at base[row * C + c]; the whole CTA syncs
template <class P, int C>
struct ColSmem {
    typename P::S* base;
    int c;
    __device__ __forceinline__ void put(int row, cx<typename P::R> v) { base[row * C + c] = P::pack(v); }
    __device__ __forceinline__ cx<typename P::R> get(int row) const { return P::load(base[row * C + c]); }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// one line per group of threads inside a warp; one pad slot every 8 avoids bank conflicts
template <class P>
struct LineSmem {
    typename P::S* base;
    static __device__ __forceinline__ int pad(int i) { return i + (i >> 3); }
    __device__ __forceinline__ void put(int i, cx<typename P::R> v) { base[pad(i)] = P::pack(v); }
    __device__ __forceinline__ cx<typename P::R> get(int i) const { return P::load(base[pad(i)]); }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
};

// one line's exchange space when a line may be wider than a warp (WIDE): such a line
// synchronises its own warps on named barrier `bar` (1..15; nthreads of them), so the
// lines of a CTA stay independent of one another
template <class P, bool WIDE>
struct LineSmemX {
    typename P::S* base;
    unsigned bar, nthreads;
    static __device__ __forceinline__ int pad(int i) { return i + (i >> 3); }
    __device__ __forceinline__ void put(int i, cx<typename P::R> v) { base[pad(i)] = P::pack(v); }
    __device__ __forceinline__ cx<typename P::R> get(int i) const { return P::load(base[pad(i)]); }
    __device__ __forceinline__ void sync() const {
        if (WIDE) asm volatile("bar.sync %0, %1;\n" ::"r"(bar), "r"(nthreads) : "memory");
        else __syncwarp();
    }
};

// ---------------------------------------------------------------------------
// Stockham stage STAGE of a length-n transform.  Butterfly b (= j + T q) of a
// radix-R stage with span Ns reads x[b + r n/R], applies exp(sg 2 pi i k r/(Ns R))
// (k = b mod Ns), takes the R-point DFT and writes y[(b - k) R + k + r Ns].
// twmul: table length / n.
// ---------------------------------------------------------------------------
template <class P, int n, int STAGE, class SM, bool TWPOW = false, bool REMFIRST = false, bool NORMLAST = true,
          bool PROT = true>
__device__ __forceinline__ void fft_stage(cx<typename P::R> (&v)[8], int j, const typename P::S* __restrict__ tw,
                                          int twmul, SM& sm, int sg) {
    typedef cx<typename P::R> C;
    typedef FftShape<n, REMFIRST> Sh;
    constexpr int RADIX = Sh::radix(STAGE);
    constexpr int Ns = Sh::span(STAGE);
    constexpr int T = Sh::T;
    constexpr int Q = 8 / RADIX;
    constexpr bool LAST = (STAGE == Sh::stages - 1);
    C out[8];
#pragma unroll
    for (int q = 0; q < Q; q++) {
        const int b = j + T * q;
        const int k = b & (Ns - 1);
        C u[RADIX];
#pragma unroll
        for (int r = 0; r < RADIX; r++) u[r] = v[q + r * Q];
        if (Ns > 1) {
            if constexpr (TWPOW && RADIX == 8) {
                // one twiddle load per butterfly, the other six powers formed on the FMA
                // pipe with at most three products in a chain (for a pass bound by the
                // L1TEX pipe that the table loads go through)
                const C w1 = twiddle<P>(tw, k * (n / (Ns * RADIX)) * twmul, sg);
                const C w2 = cmul(w1, w1), w3 = cmul(w2, w1), w4 = cmul(w2, w2);
                const C w5 = cmul(w4, w1), w6 = cmul(w4, w2), w7 = cmul(w4, w3);
                u[1] = P::ctw(u[1], w1);
                u[2] = P::ctw(u[2], w2);
                u[3] = P::ctw(u[3], w3);
                u[4] = P::ctw(u[4], w4);
                u[5] = P::ctw(u[5], w5);
                u[6] = P::ctw(u[6], w6);
                u[7] = P::ctw(u[7], w7);
            } else if constexpr (TWPOW && RADIX == 4) {
                const C w1 = twiddle<P>(tw, k * (n / (Ns * RADIX)) * twmul, sg);
                const C w2 = cmul(w1, w1), w3 = cmul(w2, w1);
                u[1] = P::ctw(u[1], w1);
                u[2] = P::ctw(u[2], w2);
                u[3] = P::ctw(u[3], w3);
            } else {
#pragma unroll
                for (int r = 1; r < RADIX; r++)
                    u[r] = P::ctw(u[r], twiddle<P>(tw, k * r * (n / (Ns * RADIX)) * twmul, sg));
            }
        }
        dft<P, RADIX, LAST && NORMLAST, PROT>(u, sg);
        if (LAST) {
#pragma unroll
            for (int r = 0; r < RADIX; r++) out[q + r * Q] = u[r];
        } else {
            const int base = (b - k) * RADIX + k;
#pragma unroll
            for (int r = 0; r < RADIX; r++) sm.put(base + r * Ns, u[r]);
        }
    }
    if (LAST) {
#pragma unroll
        for (int s = 0; s < 8; s++) v[s] = out[s];
    } else {
        sm.sync();
#pragma unroll
        for (int s = 0; s < 8; s++) v[s] = sm.get(j + T * s);
        sm.sync();
    }
}

// full length-n transform, unnormalised, sign sg; in and out: v[s] = x[j + T s].
// TWPOW: radix-8 stages form the twiddle powers by products instead of table loads;
// REMFIRST: the short stage first (FftShape); NORMLAST = false leaves the double-float
// outputs unnormalised too, for consumers that take lazy sums of them or convert both
// words exactly (everything but the statistics of u, which read the high word)
template <class P, int n, class SM, bool TWPOW = false, bool REMFIRST = false, bool NORMLAST = true, bool PROT = true>
__device__ __forceinline__ void fft(cx<typename P::R> (&v)[8], int j, const typename P::S* __restrict__ tw, int twmul,
                                    SM& sm, int sg) {
    typedef FftShape<n, REMFIRST> Sh;
    fft_stage<P, n, 0, SM, TWPOW, REMFIRST, NORMLAST, PROT>(v, j, tw, twmul, sm, sg);
    if constexpr (Sh::stages > 1) fft_stage<P, n, 1, SM, TWPOW, REMFIRST, NORMLAST, PROT>(v, j, tw, twmul, sm, sg);
    if constexpr (Sh::stages > 2) fft_stage<P, n, 2, SM, TWPOW, REMFIRST, NORMLAST, PROT>(v, j, tw, twmul, sm, sg);
    if constexpr (Sh::stages > 3) fft_stage<P, n, 3, SM, TWPOW, REMFIRST, NORMLAST, PROT>(v, j, tw, twmul, sm, sg);
}

// ---------------------------------------------------------------------------
// value conversion between precisions (only FP64 -> any is needed)
// ---------------------------------------------------------------------------
template <class Pfrom, class Pto>
struct Convert;
template <class P>
struct Convert<P, P> {
    static __device__ __forceinline__ cx<typename P::R> go(cx<typename P::R> c) { return c; }
};
template <>
struct Convert<PrecF64, PrecDF> {
    static __device__ __forceinline__ cx<df> go(cx<double> c) { return cmake<df>(d2df_int(c.re), d2df_int(c.im)); }
};
template <>
struct Convert<PrecF64, PrecF32> {
    static __device__ __forceinline__ cx<float> go(cx<double> c) { return cmake<float>(d2f_int(c.re), d2f_int(c.im)); }
};
template <>
struct Convert<PrecDF, PrecF64> {   // exact conversions of the two words, one FP64 add each
    static __device__ __forceinline__ cx<double> go(cx<df> c) {
        return cmake<double>(f2d_int(c.re.hi) + f2d_int(c.re.lo), f2d_int(c.im.hi) + f2d_int(c.im.lo));
    }
};

// ---------------------------------------------------------------------------
// per-thread statistics of u on the x pass: sum u^4 and max |u|
// ---------------------------------------------------------------------------
struct NSum {  // Neumaier pair
    double s, c;
    __device__ __forceinline__ void add(double x) {
        double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ double value() const { return s + c; }
};

template <class P>
struct Stats;

template <>
struct Stats<PrecF64> {
    NSum sum;
    unsigned long long mx;
    __device__ __forceinline__ void init() { sum.s = 0.0; sum.c = 0.0; mx = 0ull; }
    __device__ __forceinline__ void take(double u, bool want_sum) {
        unsigned long long key = (unsigned long long)__double_as_longlong(u) & 0x7FFFFFFFFFFFFFFFull;
        mx = key > mx ? key : mx;
        if (want_sum) {
            double u2 = u * u;
            sum.add(u2 * u2);
        }
    }
    // complex field: m2 = |u|^2 >= 0; the key is |u|^2 and the sum takes |u|^4
    __device__ __forceinline__ void take_sq(double m2, bool want_sum) {
        const unsigned long long key = (unsigned long long)__double_as_longlong(m2);
        mx = key > mx ? key : mx;
        if (want_sum) sum.add(m2 * m2);
    }
    __device__ __forceinline__ void take2(cx<double> u, bool want_sum) {
        take(u.re, want_sum);
        take(u.im, want_sum);
    }
    __device__ __forceinline__ double total() const { return sum.value(); }
    __device__ __forceinline__ double maxval() const { return __longlong_as_double((long long)mx); }
    // float bits of max|u| (nan above inf above every finite value)
    __device__ __forceinline__ unsigned fkey() const {
        return __float_as_uint(d2f_int(__longlong_as_double((long long)mx))) & 0x7FFFFFFFu;
    }
    // bits of max|u| as a double: unsigned order = numeric order, nan above inf
    __device__ __forceinline__ unsigned long long dkey() const { return mx; }
};

template <>
struct Stats<PrecDF> {
    df acc;
    dfc acc2;   // the sums of take2, one per lane, unnormalised (non-negative terms)
    unsigned int mx;
    __device__ __forceinline__ void init() {
        acc = df_make(0.f, 0.f);
        acc2.h = acc2.l = make_float2(0.f, 0.f);
        mx = 0u;
    }
    // u may be unnormalised: the key is the float nearest hi + lo
    __device__ __forceinline__ void take(df u, bool want_sum) {
        unsigned int key = __float_as_uint(__fadd_rn(u.hi, u.lo)) & 0x7FFFFFFFu;
        mx = key > mx ? key : mx;
        if (want_sum) {
            df u2 = u * u;
            acc = acc + u2 * u2;
        }
    }
    // both components of u at once (the two lines of a pair), on packed FP32x2 pairs
    __device__ __forceinline__ void take2(cx<df> u, bool want_sum) {
        const dfc x = PrecDF::split(u);
        const float2 r = f2add(x.h, x.l);
        const unsigned k0 = __float_as_uint(r.x) & 0x7FFFFFFFu, k1 = __float_as_uint(r.y) & 0x7FFFFFFFu;
        mx = k0 > mx ? k0 : mx;
        mx = k1 > mx ? k1 : mx;
        if (want_sum) {
            const dfc u2 = dfc_mul_lazy(x, x);
            acc2 = dfc_add_lazy(acc2, dfc_mul_lazy(u2, u2));
        }
    }
    // complex field: m2 = |u|^2 >= 0; the key is |u|^2 and the sum takes |u|^4
    __device__ __forceinline__ void take_sq(df m2, bool want_sum) {
        const unsigned int key = __float_as_uint(m2.hi);
        mx = key > mx ? key : mx;
        if (want_sum) acc = acc + m2 * m2;
    }
    __device__ __forceinline__ double total() const {
        return (f2d_int(acc.hi) + f2d_int(acc.lo)) + ((f2d_int(acc2.h.x) + f2d_int(acc2.l.x)) +
                                                      (f2d_int(acc2.h.y) + f2d_int(acc2.l.y)));
    }
    // the same sum as a double-float (unnormalised; every term is non-negative)
    __device__ __forceinline__ df total_df() const {
        return df_add_lazy(acc, df_add_lazy(df_make(acc2.h.x, acc2.l.x), df_make(acc2.h.y, acc2.l.y)));
    }
    __device__ __forceinline__ double maxval() const { return f2d_int(__uint_as_float(mx)); }
    __device__ __forceinline__ unsigned fkey() const { return mx; }
    __device__ __forceinline__ unsigned long long dkey() const {
        return (unsigned long long)__double_as_longlong(f2d_int(__uint_as_float(mx)));
    }
};

template <>
struct Stats<PrecF32> {
    df acc;
    unsigned int mx;
    __device__ __forceinline__ void init() { acc = df_make(0.f, 0.f); mx = 0u; }
    __device__ __forceinline__ void take(float u, bool want_sum) {
        unsigned int key = __float_as_uint(u) & 0x7FFFFFFFu;
        mx = key > mx ? key : mx;
        if (want_sum) {
            float u2 = u * u;
            acc = acc + df_make(u2 * u2, 0.f);
        }
    }
    __device__ __forceinline__ void take2(cx<float> u, bool want_sum) {
        take(u.re, want_sum);
        take(u.im, want_sum);
    }
    __device__ __forceinline__ void take_sq(float m2, bool want_sum) {
        const unsigned int key = __float_as_uint(m2);
        mx = key > mx ? key : mx;
        if (want_sum) acc = acc + df_make(m2 * m2, 0.f);
    }
    __device__ __forceinline__ double total() const { return f2d_int(acc.hi) + f2d_int(acc.lo); }
    __device__ __forceinline__ double maxval() const { return f2d_int(__uint_as_float(mx)); }
    __device__ __forceinline__ unsigned fkey() const { return mx; }
    __device__ __forceinline__ unsigned long long dkey() const {
        return (unsigned long long)__double_as_longlong(f2d_int(__uint_as_float(mx)));
    }
};

// ---------------------------------------------------------------------------
// device-side run state (lives in device memory; read by the passes so that a
// captured step needs no host decisions)
// ---------------------------------------------------------------------------
struct KgDev {
    long long level;          // n
    int phase;                // 0: S0 = uh^n, S1 = uh^{n-1}; 1: swapped
    int frozen;               // blow-up flag
    long long blowup_level;   // level at which the state froze
    int energy_every;         // record Q, P on steps from level l with (l+1) % energy_every == 0
    int complex_field;        // 1: complex u; the x pass max keys are |u|^2
    double threshold;         // > 0: blow-up check max|u^n| > threshold
    double maxabs_last;       // max |u^l| of the last x pass of a step
    double P_last;            // P^l of the last recording step
    long long P_last_level;
    double Q_last;            // Q^{l+1/2} of the last recording step
    long long Q_last_level;
    double P_peek;            // sum-based P of the last peek
    double maxabs_peek;
    int status;               // nonzero: a device-side check failed
    int scheme;               // KG_SCHEME_EQ2 (0) or KG_SCHEME_COMPOSED4 (1)
    int sub;                  // composed scheme: substep 0..2 of the current step
    int record_p;             // 1: the next x pass records P^l whatever energy_every says (cleared by k_fin_x)
};

__device__ __forceinline__ bool kg_recording(const KgDev* dev) {
    return dev->energy_every > 0 && ((dev->level + 1) % dev->energy_every) == 0;
}

// ---------------------------------------------------------------------------
// block reduction of (Neumaier pair, max) -> thread 0
// ---------------------------------------------------------------------------
__device__ __forceinline__ void nsum_merge(NSum& a, const NSum& b) {
    a.add(b.s);
    a.c += b.c;
}

// maximum of 64-bit keys over a CTA of NT threads (a power of two) -> thread 0
template <int NT>
__device__ __forceinline__ unsigned long long block_max_key(unsigned long long k, unsigned long long* sh) {
    constexpr unsigned kMask = NT >= 32 ? 0xffffffffu : ((1u << NT) - 1u);
    constexpr int kOff0 = NT >= 32 ? 16 : NT / 2;
#pragma unroll
    for (int o = kOff0; o > 0; o >>= 1) {
        const unsigned long long b = __shfl_down_sync(kMask, k, o);
        k = b > k ? b : k;
    }
    constexpr int NW = (NT + 31) / 32;
    if (NW > 1) {
        __syncthreads();
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = k;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int w = 1; w < NW; w++) k = sh[w] > k ? sh[w] : k;
    }
    return k;
}

// NT threads, a power of two; lane 0 of warp 0 ends with the block result
// sum of one non-negative double-float value per thread of an NT-thread CTA on the FP32
// pipe (unnormalised sums; the FP64 Neumaier reduction of block_reduce spends most of a
// recording x pass's extra time in its dependent FP64 chain); the total lands in thread 0
template <int NT>
__device__ __forceinline__ df block_sum_df(df v, df* sm) {
    static_assert(NT % 32 == 0 && NT <= 1024, "whole warps");
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = df_add_lazy(v, df_make(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sm[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < NT / 32 ? sm[l] : df_make(0.f, 0.f);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v = df_add_lazy(v, df_make(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)));
    }
    return v;
}

template <int NT>
__device__ __forceinline__ void block_reduce(NSum& v, double& mx, double* sh) {
    // sh: 3 * 32 doubles
    constexpr unsigned kMask = NT >= 32 ? 0xffffffffu : ((1u << NT) - 1u);
    constexpr int kOff0 = NT >= 32 ? 16 : NT / 2;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = kOff0; o > 0; o >>= 1) {
        NSum b;
        b.s = __shfl_down_sync(kMask, v.s, o);
        b.c = __shfl_down_sync(kMask, v.c, o);
        double m = __shfl_down_sync(kMask, mx, o);
        nsum_merge(v, b);
        mx = (m > mx || m != m) ? m : mx;
    }
    constexpr int NW = (NT + 31) / 32;
    if (NW > 1) {
        __syncthreads();
        if (lane == 0) {
            sh[w] = v.s;
            sh[32 + w] = v.c;
            sh[64 + w] = mx;
        }
        __syncthreads();
        if (w == 0) {
            NSum t;
            t.s = lane < NW ? sh[lane] : 0.0;
            t.c = lane < NW ? sh[32 + lane] : 0.0;
            double m = lane < NW ? sh[64 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                NSum b;
                b.s = __shfl_down_sync(0xffffffffu, t.s, o);
                b.c = __shfl_down_sync(0xffffffffu, t.c, o);
                double mm = __shfl_down_sync(0xffffffffu, m, o);
                nsum_merge(t, b);
                m = (mm > m || mm != mm) ? mm : m;
            }
            v = t;
            mx = m;
        }
    }
}

}  // namespace kg
