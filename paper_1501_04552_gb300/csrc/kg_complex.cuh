// kg_complex.cuh -- x-direction kernels for a complex field u (section 1.1.2: the
// paper's implementation allows a complex field; Eq. (1) has the nonlinearity |u|^2 u).
//
// The spectrum is the full N^3 array [kz][ky][kx] (kx = 0..N-1 in FFT order), so the
// x direction is a plain complex transform of N points per line: no real-to-complex
// packing, no C2R rule.  The y and z passes are the column kernels of the real field
// with N columns per plane instead of N/2 + 1.
#pragma once
#include "kg_kernels.cuh"

namespace kg {

template <int N>
struct XcShape {
    static constexpr int T = N / 8;             // threads per x-line
    static constexpr int LPC = kXThreads / T;   // lines per CTA
    static constexpr int PADN = N + N / 8;      // padded shared-memory slots per line
    static constexpr bool CTA_SYNC = T > 32;    // a line spans more than one warp
    static_assert(kXThreads % T == 0, "whole lines per CTA");
    static_assert(!CTA_SYNC || LPC <= 15, "one named barrier per line");
};

// resident CTAs per SM the complex x pass is compiled for (the largest count whose
// register budget needs no spills, FP64 excepted)
template <class P>
struct XcMinBlocks {
    static constexpr int value = 4;
};
template <>
struct XcMinBlocks<PrecF64> {
    static constexpr int value = 2;
};

// Pass X of a complex field.  MODE_STEP: per x-line, inverse transform, scale 1/N^3 ->
// u^n; |u|^2 keys and (when wanted) sum |u|^4; F = lam |u|^2 u; forward transform;
// written back in place.  MODE_PEEK: inverse transform and the statistics only.
template <class P, int N, int MODE>
__global__ void __launch_bounds__(kXThreads, XcMinBlocks<P>::value) k_pass_xc(typename P::S* __restrict__ W, KgDev* __restrict__ dev,
                                                         double* __restrict__ part_sum, double* __restrict__ part_max,
                                                         const typename P::S* __restrict__ tw, double scale,
                                                         double lam) {
    typedef typename P::S S;
    typedef typename P::R R;
    typedef cx<R> C;
    typedef XcShape<N> X;
    constexpr int T = X::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    S* sm = reinterpret_cast<S*>(smraw);
    __shared__ double red[96];

    const int li = threadIdx.x / T, j = threadIdx.x % T;
    const size_t line = (size_t)blockIdx.x * X::LPC + li;
    LineSmemX<P, X::CTA_SYNC> lsm{sm + li * X::PADN, 1u + (unsigned)li, (unsigned)T};
    const bool want_sum = (MODE == MODE_PEEK) || kg_recording(dev) || dev->record_p;
    const R rlam = P::from_f64(lam);
    S* __restrict__ L = W + line * N;
    Stats<P> st;
    st.init();

    C v[8];
#pragma unroll
    for (int s = 0; s < 8; s++) v[s] = P::load(L[j + T * s]);
    // inverse transform, then (stepping pass) the forward one, through one copy of the code
#pragma unroll 1
    for (int dir = 0; dir < (MODE == MODE_STEP ? 2 : 1); dir++) {
        // FP32: twiddle powers by products (the pass is bound by the L1TEX pipe)
        fft<P, N, LineSmemX<P, X::CTA_SYNC>, sizeof(R) == 4>(v, j, tw, 1, lsm, dir == 0 ? +1 : -1);
        if (dir == 0) {
#pragma unroll
            for (int s = 0; s < 8; s++) {
                v[s].re = P::scale2(v[s].re, scale);   // scale = 1/N^3, a power of two
                v[s].im = P::scale2(v[s].im, scale);
                const R m2 = v[s].re * v[s].re + v[s].im * v[s].im;
                st.take_sq(m2, want_sum);
                if (MODE == MODE_STEP) {
                    const R g = rlam * m2;
                    v[s].re = g * v[s].re;
                    v[s].im = g * v[s].im;
                }
            }
        }
    }
    if (MODE == MODE_STEP) {
#pragma unroll
        for (int s = 0; s < 8; s++) L[j + T * s] = P::pack(v[s]);
    }

    __shared__ unsigned long long kred[kXThreads / 32];
    const unsigned long long key = block_max_key<kXThreads>(st.dkey(), kred);
    if (threadIdx.x == 0) part_max[blockIdx.x] = __longlong_as_double((long long)key);
    if (want_sum) {
        NSum acc;
        acc.s = st.total();
        acc.c = 0.0;
        double unused = 0.0;
        block_reduce<kXThreads>(acc, unused, red);
        if (threadIdx.x == 0) part_sum[blockIdx.x] = acc.value();
    }
}

// Set-up and read-out along x of a complex field in the pass precision, one line per N/8
// threads: FWD: complex FP64 lines u_in (lam |u|^2 u when cube) -> their transforms,
// unnormalised, in spec (pass precision); else spec -> lines times scale, FP64, into u_out.
template <class P, int N, bool FWD>
__global__ void __launch_bounds__(kXThreads) k_xc_io(const double2* __restrict__ u_in, typename P::S* __restrict__ spec,
                                                     double2* __restrict__ u_out,
                                                     const typename P::S* __restrict__ tw, int cube, double lam,
                                                     double scale) {
    typedef typename P::R R;
    typedef cx<R> C;
    typedef XcShape<N> X;
    constexpr int T = X::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    typename P::S* sm = reinterpret_cast<typename P::S*>(smraw);
    const int li = threadIdx.x / T, j = threadIdx.x % T;
    const size_t line = (size_t)blockIdx.x * X::LPC + li;
    LineSmemX<P, X::CTA_SYNC> lsm{sm + li * X::PADN, 1u + (unsigned)li, (unsigned)T};
    typename P::S* __restrict__ Ls = spec + line * N;
    C v[8];
    if constexpr (FWD) {
        const R rlam = P::from_f64(lam);
#pragma unroll
        for (int s = 0; s < 8; s++) {
            const double2 z = u_in[line * N + j + T * s];
            v[s] = Convert<PrecF64, P>::go(cmake<double>(z.x, z.y));
            if (cube) {
                const R g = rlam * (v[s].re * v[s].re + v[s].im * v[s].im);
                v[s].re = g * v[s].re;
                v[s].im = g * v[s].im;
            }
        }
        fft<P, N>(v, j, tw, 1, lsm, -1);
#pragma unroll
        for (int s = 0; s < 8; s++) Ls[j + T * s] = P::pack(v[s]);
    } else {
#pragma unroll
        for (int s = 0; s < 8; s++) v[s] = P::load(Ls[j + T * s]);
        fft<P, N>(v, j, tw, 1, lsm, +1);
#pragma unroll
        for (int s = 0; s < 8; s++) {
            const cx<double> w = Convert<P, PrecF64>::go(
                cmake<R>(P::scale2(v[s].re, scale), P::scale2(v[s].im, scale)));
            u_out[line * N + j + T * s] = make_double2(w.re, w.im);
        }
    }
}

// FP64 set-up: forward transform along x of complex physical lines,
// out[line][k] = sum_x f(u[line][x]) e^{-2 pi i k x / N}, f(u) = u or lam |u|^2 u
template <int N>
__global__ void __launch_bounds__(kXThreads) k_xc_forward(const double2* __restrict__ u, double2* __restrict__ out,
                                                          const double2* __restrict__ tw, int cube, double lam) {
    typedef PrecF64 P;
    typedef XcShape<N> X;
    constexpr int T = X::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    double2* sm = reinterpret_cast<double2*>(smraw);
    const int li = threadIdx.x / T, j = threadIdx.x % T;
    const size_t line = (size_t)blockIdx.x * X::LPC + li;
    LineSmemX<P, X::CTA_SYNC> lsm{sm + li * X::PADN, 1u + (unsigned)li, (unsigned)T};
    cx<double> v[8];
#pragma unroll
    for (int s = 0; s < 8; s++) {
        double2 z = u[line * N + j + T * s];
        if (cube) {
            const double g = lam * (z.x * z.x + z.y * z.y);
            z = make_double2(g * z.x, g * z.y);
        }
        v[s] = cmake<double>(z.x, z.y);
    }
    fft<P, N>(v, j, tw, 1, lsm, -1);
#pragma unroll
    for (int s = 0; s < 8; s++) out[line * N + j + T * s] = make_double2(v[s].re, v[s].im);
}

// FP64 read-out: inverse transform along x, times scale, into u (may be NULL);
// optionally the per-CTA sum of |u|^4
template <int N>
__global__ void __launch_bounds__(kXThreads) k_xc_inverse(const double2* __restrict__ in, double2* __restrict__ u,
                                                          const double2* __restrict__ tw, double scale,
                                                          double* __restrict__ part_sum) {
    typedef PrecF64 P;
    typedef XcShape<N> X;
    constexpr int T = X::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    double2* sm = reinterpret_cast<double2*>(smraw);
    __shared__ double red[96];
    const int li = threadIdx.x / T, j = threadIdx.x % T;
    const size_t line = (size_t)blockIdx.x * X::LPC + li;
    LineSmemX<P, X::CTA_SYNC> lsm{sm + li * X::PADN, 1u + (unsigned)li, (unsigned)T};
    cx<double> v[8];
#pragma unroll
    for (int s = 0; s < 8; s++) {
        const double2 z = in[line * N + j + T * s];
        v[s] = cmake<double>(z.x, z.y);
    }
    fft<P, N>(v, j, tw, 1, lsm, +1);
    NSum acc;
    acc.s = 0.0;
    acc.c = 0.0;
#pragma unroll
    for (int s = 0; s < 8; s++) {
        const double a = v[s].re * scale, b = v[s].im * scale;
        if (u) u[line * N + j + T * s] = make_double2(a, b);
        if (part_sum) {
            const double m2 = a * a + b * b;
            acc.add(m2 * m2);
        }
    }
    if (part_sum) {
        double mx = 0.0;
        block_reduce<kXThreads>(acc, mx, red);
        if (threadIdx.x == 0) part_sum[blockIdx.x] = acc.value();
    }
}

}  // namespace kg
