// kg_kernels.cuh -- kernel templates of the step passes, the set-up and the read-out.
#pragma once
#include <type_traits>
#include "kg_fft.cuh"
#include "kg_launch.h"

namespace kg {

// ---------------------------------------------------------------------------
// Pass X.  MODE_STEP: C2R along x, stats, F = lam u^3, R2C along x, in place.
//          MODE_PEEK: C2R along x and stats only (W untouched).
// One line = N/2+1 complex values; T = N/16 threads per line, 256 threads per CTA.
// ---------------------------------------------------------------------------
constexpr int kXThreads = 256;

template <int N>
struct XShape {
    static constexpr int M = N / 2;
    static constexpr int T = M / 8;
    static constexpr int LPC = kXThreads / T;           // lines per CTA
    static constexpr int PADM = M + M / 8;              // padded smem slots per line
    static_assert(T <= 32, "one line must fit in a warp");
};

// LIN: a pointer to the line's N/2+1 values, or any type whose operator[] yields them
// (the cluster-fused pass reads lines spread over the shared memory of several CTAs)
template <class P, int N, class LIN = const typename P::S*>
__device__ __forceinline__ void x_load_c2r(LIN line, int j, const typename P::S* __restrict__ tw,
                                           cx<typename P::R> (&v)[8]) {
    typedef typename P::R R;
    typedef cx<R> C;
    constexpr int M = N / 2, T = XShape<N>::T;
    constexpr bool kPow = sizeof(R) == 4;   // FP32: twiddles by products (L1TEX-bound pass)
    C wr[8];
    if constexpr (kPow) twiddle_run<P>(tw, j, T, +1, wr);
#pragma unroll
    for (int s = 0; s < 8; s++) {
        const int k = j + T * s;
        C X = P::load(line[k]);
        C Xp = P::load(line[M - k]);       // k = 0 pairs with the Nyquist entry k = M
        if (k == 0) {                      // real parts only at kx = 0 and kx = N/2
            X.im = P::from_f64(0.0);
            Xp.im = P::from_f64(0.0);
        }
        C A = P::cadd(X, conj(Xp));
        C B = P::csub(X, conj(Xp));
        C Bw;                                                // B exp(+2 pi i k / N)
        if constexpr (kPow) Bw = P::ctw(B, wr[s]);
        else Bw = P::ctw(B, twiddle<P>(tw, k, +1));
        v[s] = P::cnorm(P::cadd(A, mul_i(Bw)));
    }
}

// One x-line (T = N/16 threads, thread j): C2R, scale, stats, and in MODE_STEP the
// cube, R2C and write-back.  The line is read from Lin (global memory, or the line's
// landing slot in shared memory, which may be lsm's own storage) and written to L
// (pointers, or element accessors as for x_load_c2r; every read precedes every write).
template <class P, int N, int MODE, class LIN = const typename P::S*, class LOUT = typename P::S* __restrict__,
          bool RF = false>
__device__ __forceinline__ void x_line_body(LIN Lin, LOUT L, int j,
                                            LineSmem<P>& lsm, const typename P::S* __restrict__ tw, double scale,
                                            typename P::R rlam, bool want_sum, Stats<P>& st) {
    typedef typename P::R R;
    typedef cx<R> C;
    constexpr int M = N / 2, T = XShape<N>::T;
    C v[8];
    x_load_c2r<P, N, LIN>(Lin, j, tw, v);
    lsm.sync();   // every lane has read Lin before the first exchange writes lsm
    // inverse transform, then (stepping pass) the forward one, through one copy of the code
#pragma unroll 1
    for (int dir = 0; dir < (MODE == MODE_STEP ? 2 : 1); dir++) {
        // the FP32 x pass is bound by the L1TEX pipe: twiddle powers by products there
        fft<P, M, LineSmem<P>, sizeof(typename P::R) == 4, RF>(v, j, tw, 2, lsm, dir == 0 ? +1 : -1);
        if (dir == 0) {
#pragma unroll
            for (int s = 0; s < 8; s++) {
                v[s].re = P::scale2(v[s].re, scale);   // scale = 1/N^3, a power of two
                v[s].im = P::scale2(v[s].im, scale);
                st.take(v[s].re, want_sum);
                st.take(v[s].im, want_sum);
            }
            if (MODE == MODE_STEP) {
#pragma unroll
                for (int s = 0; s < 8; s++) {
                    v[s].re = rlam * (v[s].re * v[s].re * v[s].re);
                    v[s].im = rlam * (v[s].im * v[s].im * v[s].im);
                }
            }
        }
    }
    if (MODE == MODE_STEP) {
        // real-to-complex post-processing: X[k] = (Z_k + conj Z_{M-k})/2 - i W^k (Z_k - conj Z_{M-k})/2
#pragma unroll
        for (int s = 0; s < 8; s++) lsm.put(j + T * s, v[s]);
        lsm.sync();
        const double half = 0.5;
        constexpr bool kPow = sizeof(R) == 4;
        C wf[8];
        if constexpr (kPow) twiddle_run<P>(tw, j, T, -1, wf);
#pragma unroll
        for (int s = 0; s < 8; s++) {
            const int k = j + T * s;
            C Z = v[s];
            C Zp = lsm.get((M - k) & (M - 1));
            C A = P::cadd(Z, conj(Zp));
            C B = P::csub(Z, conj(Zp));
            C D;                                                // i B exp(-2 pi i k / N)
            if constexpr (kPow) D = mul_i(P::ctw(B, wf[s]));
            else D = mul_i(P::ctw(B, twiddle<P>(tw, k, -1)));
            C out = P::cnorm(P::csub(A, D));
            out.re = P::scale2(out.re, half);
            out.im = P::scale2(out.im, half);
            L[k] = P::pack(out);
            if (k == 0) L[M] = P::pack(cmake<R>(Z.re - Z.im, P::from_f64(0.0)));
        }
        lsm.sync();
    }
}

// Two x-lines of a real field through one N-point complex transform.  Over the Hermitian
// extensions of both half spectra (real parts only at kx = 0 and N/2, the C2R rule),
// Z[k] = X1[k] + i X2[k] has the inverse transform u1 + i u2; after the cube, the forward
// transform of F1 + i F2 splits again as
//     X1[k] = (Z[k] + conj Z[N-k]) / 2,    X2[k] = -i (Z[k] - conj Z[N-k]) / 2,
// which needs no twiddle product (the one-line form packs each line into an N/2-point
// transform with a twiddle product per point on the way in and on the way out).
template <int N>
struct XpShape {
    static constexpr int T = N / 8;              // threads per line pair
    static constexpr int PPC = kXThreads / T;    // pairs per CTA
    static constexpr int PADN = N + N / 8;       // padded exchange slots per pair
    static constexpr bool CTA_SYNC = T > 32;     // a pair spans more than one warp
    static_assert(2 * PPC == XShape<N>::LPC && PPC * PADN == XShape<N>::LPC * XShape<N>::PADM,
                  "same lines and shared memory per CTA as the one-line form");
    static_assert(!CTA_SYNC || PPC <= 15, "one named barrier per pair");
};

// v[s] = X1[k] + i X2[k], k = j + T s, from the half spectra L1, L2 of two x-lines
// (Hermitian extension; the kx = 0 and N/2 entries contribute their real parts)
template <class P, int N>
__device__ __forceinline__ void x_pair_load(const typename P::S* __restrict__ L1, const typename P::S* __restrict__ L2,
                                            int j, cx<typename P::R> (&v)[8]) {
    typedef typename P::R R;
    typedef cx<R> C;
    constexpr int T = N / 8;
    const R zero = P::from_f64(0.0);
#pragma unroll
    for (int s = 0; s < 8; s++) {
        const int k = j + T * s;
        const int kk = k <= N / 2 ? k : N - k;
        C X1 = P::load(L1[kk]), X2 = P::load(L2[kk]);
        if (kk == 0 || kk == N / 2) {      // real parts only
            X1.im = zero;
            X2.im = zero;
        }
        if (k > N / 2) {                    // Hermitian extension
            X1 = conj(X1);
            X2 = conj(X2);
        }
        // X1 + i X2, left unnormalised: the transform's first stage takes lazy sums of it
        v[s] = P::cadd_i(X1, X2);
    }
}

// the half spectra of two real lines from Z = FFT(x1 + i x2) held as v[s] = Z[j + T s]:
// X1 = (Z + conj Zm) / 2, X2 = -i (Z - conj Zm) / 2, Zm the mirrored entry
template <class P, int N, class SM>
__device__ __forceinline__ void x_pair_unpack(typename P::S* __restrict__ L1, typename P::S* __restrict__ L2, int j,
                                              SM& lsm, const cx<typename P::R> (&v)[8]) {
    typedef typename P::R R;
    typedef cx<R> C;
    constexpr int T = N / 8;
#pragma unroll
    for (int s = 0; s < 8; s++) lsm.put(j + T * s, v[s]);
    lsm.sync();
#pragma unroll
    for (int s = 0; s < 8; s++) {
        const int k = j + T * s;
        if (k <= N / 2) {
            const C Z = v[s];
            const C Zm = conj(lsm.get((N - k) & (N - 1)));
            const C A = P::cadd(Z, Zm), B = P::csub(Z, Zm);      // 2 X1, 2 i X2
            // stored unnormalised: every reader of W starts with lazy sums or an exact
            // conversion of both words
            L1[k] = P::pack(P::cscale2(A, 0.5));
            L2[k] = P::pack(P::cscale2(P::cmul_negi(B), 0.5));
        }
    }
    lsm.sync();
}

template <class P, int N, int MODE, class SM, bool RF = false>
__device__ __forceinline__ void x_pair_body(typename P::S* __restrict__ L1, int j, SM& lsm,
                                            const typename P::S* __restrict__ tw, double scale, typename P::R rlam,
                                            bool want_sum, Stats<P>& st) {
    typedef typename P::R R;
    typedef cx<R> C;
    constexpr int NH = N / 2 + 1;
    typename P::S* __restrict__ L2 = L1 + NH;
    C v[8];
    x_pair_load<P, N>(L1, L2, j, v);
#pragma unroll 1
    for (int dir = 0; dir < (MODE == MODE_STEP ? 2 : 1); dir++) {
        // outputs left unnormalised: the statistics read the rounded sum of both words, the
        // cube and the unpacking take lazy products and sums
        fft<P, N, SM, false, RF, false>(v, j, tw, 1, lsm, dir == 0 ? +1 : -1);
        if (dir == 0) {
#pragma unroll
            for (int s = 0; s < 8; s++) {
                v[s].re = P::scale2(v[s].re, scale);   // u1, u2 at x = j + T s; scale = 1/N^3
                v[s].im = P::scale2(v[s].im, scale);
                st.take2(v[s], want_sum);
            }
            if (MODE == MODE_STEP) {
#pragma unroll
                for (int s = 0; s < 8; s++) {
                    v[s].re = P::cube(v[s].re, rlam);
                    v[s].im = P::cube(v[s].im, rlam);
                }
            }
        }
    }
    if (MODE == MODE_STEP) x_pair_unpack<P, N>(L1, L2, j, lsm, v);
}

// one element global -> shared without registers (8- or 16-byte values)
template <class S>
__device__ __forceinline__ void cp_async_elem(S* smem, const S* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(S) == 16) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
    } else {
        static_assert(sizeof(S) == 8, "8- or 16-byte elements");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
    }
}

// The double-float and FP64 passes take x-lines in pairs (x_pair_body): fewer
// arithmetic operations per point, which is what bounds them.
template <class P>
struct XPaired {
    static constexpr bool value = false;
};
template <>
struct XPaired<PrecDF> {
    static constexpr bool value = true;
};
template <>
struct XPaired<PrecF64> {
    static constexpr bool value = true;
};

// resident CTAs per SM the x pass is compiled for: the paired double-float body fits
// four (64 registers, no spills; 1.61 -> 1.44 ms at 512^3 against two); the pipelined
// FP32 body measured slower at three (0.48 -> 0.51 ms), and the FP64 body needs its registers
template <class P>
struct XMinBlocks {
    static constexpr int value = 2;
};
template <>
struct XMinBlocks<PrecDF> {
    static constexpr int value = 4;
};

// How pass X walks W.  Pipelined (the FP32 pass, bound by latency and the L1TEX pipe): a
// persistent grid walks the batches, and while a CTA transforms one batch from shared
// memory the next one lands in the other half of a double buffer (cp.async).  Direct
// (the double-float and FP64 passes, bound by their arithmetic pipes, where the copy loop
// and the extra barriers cost more than they hide): one batch per CTA, loaded from global
// memory straight into registers.
template <class P>
struct XPipelined {
    static constexpr bool value = true;
};
template <>
struct XPipelined<PrecDF> {
    static constexpr bool value = false;
};
template <>
struct XPipelined<PrecF64> {
    static constexpr bool value = false;
};

// Pass X.  A batch is LPC consecutive x-lines, one contiguous run of LPC (N/2+1) values
// of W; a landed batch serves as the lines' FFT exchange space.  Each CTA writes one
// max key and (when wanted) one Sigma u^4 partial.
template <class P, int N, int MODE>
__global__ void __launch_bounds__(kXThreads, XMinBlocks<P>::value) k_pass_x(typename P::S* __restrict__ W, KgDev* __restrict__ dev,
                                                      double* __restrict__ part_sum, double* __restrict__ part_max,
                                                      const typename P::S* __restrict__ tw, double scale, double lam) {
    typedef typename P::S S;
    typedef XShape<N> X;
    constexpr int T = X::T, NH = N / 2 + 1, LPC = X::LPC, PADM = X::PADM;
    constexpr int NB = N * N / LPC;     // batches
    constexpr int CHUNK = LPC * NH;     // values of one batch
    static_assert(PADM >= NH, "a line lands in its exchange slot");
    extern __shared__ __align__(16) unsigned char smraw[];
    S* buf = reinterpret_cast<S*>(smraw);   // (2 when pipelined) x LPC x PADM values
    __shared__ double red[96];

    const int li = threadIdx.x / T, j = threadIdx.x % T;
    const bool want_sum = (MODE == MODE_PEEK) || kg_recording(dev) || dev->record_p;
    const typename P::R rlam = P::from_f64(lam);
    Stats<P> st;
    st.init();

    if constexpr (!XPipelined<P>::value && XPaired<P>::value) {
        typedef XpShape<N> XP;
        const int pi = threadIdx.x / XP::T, jp = threadIdx.x % XP::T;
        const size_t pair = (size_t)blockIdx.x * XP::PPC + pi;
        LineSmemX<P, XP::CTA_SYNC> lsm{buf + pi * XP::PADN, 1u + (unsigned)pi, (unsigned)XP::T};
        x_pair_body<P, N, MODE>(W + 2 * pair * NH, jp, lsm, tw, scale, rlam, want_sum, st);
    } else if constexpr (!XPipelined<P>::value) {
        const size_t line = (size_t)blockIdx.x * LPC + li;
        LineSmem<P> lsm{buf + li * PADM};
        x_line_body<P, N, MODE>(W + line * NH, W + line * NH, j, lsm, tw, scale, rlam, want_sum, st);
    } else {
        auto issue = [&](int batch, S* dst) {
            const S* src = W + (size_t)batch * CHUNK;
            for (int e = threadIdx.x; e < CHUNK; e += kXThreads) {
                const int l = e / NH;
                cp_async_elem(dst + l * PADM + (e - l * NH), src + e);
            }
        };
        int b = blockIdx.x;
        if (b < NB) issue(b, buf);
        cp_async_commit();
        for (int it = 0; b < NB; b += gridDim.x, ++it) {
            S* cur = buf + (it & 1) * (LPC * PADM);
            if (b + (int)gridDim.x < NB) issue(b + gridDim.x, buf + ((it + 1) & 1) * (LPC * PADM));
            cp_async_commit();
            cp_async_wait_1();
            __syncthreads();
            LineSmem<P> lsm{cur + li * PADM};
            x_line_body<P, N, MODE>(cur + li * PADM, W + ((size_t)b * LPC + li) * NH, j, lsm, tw, scale, rlam, want_sum,
                                    st);
            __syncthreads();   // the buffer is the target of the copy issued next iteration
        }
        cp_async_wait_all();
    }

    // the max every step (integer keys), the compensated FP64 sum only when it is wanted
    __shared__ unsigned long long kred[kXThreads / 32];
    const unsigned long long key = block_max_key<kXThreads>(st.dkey(), kred);
    if (threadIdx.x == 0) part_max[blockIdx.x] = __longlong_as_double((long long)key);
    if (want_sum) {
        if constexpr (XPaired<P>::value && !std::is_same<P, PrecF64>::value) {
            __shared__ df dred[kXThreads / 32];
            const df t = block_sum_df<kXThreads>(st.total_df(), dred);
            if (threadIdx.x == 0) part_sum[blockIdx.x] = f2d_int(t.hi) + f2d_int(t.lo);
        } else {
            NSum acc;
            acc.s = st.total();
            acc.c = 0.0;
            double unused = 0.0;
            block_reduce<kXThreads>(acc, unused, red);
            if (threadIdx.x == 0) part_sum[blockIdx.x] = acc.value();
        }
    }
}

// ---------------------------------------------------------------------------
// Column FFT: C consecutive kx columns of one plane, all N rows, in place or
// from a source array in another storage format (set-up / read-out).
// Y passes: plane = z, plane stride N*NH, row stride NH.
// Z passes: plane = ky, plane stride NH, row stride N*NH.
// ---------------------------------------------------------------------------
template <class P>
struct ColShape {
    static constexpr int C = 128 / (int)sizeof(typename P::S);
};
// Column tiles of the single-state step: 128-byte rows, except the FP32 y passes, whose
// rows are N/2+1 values apart (the z rows are a whole plane apart): there 64-byte rows
// gave twice the CTAs for the same occupancy and measured faster (0.227 against
// 0.244 ms at 512^3), while every z pass and the 16-byte y passes were as fast or faster
// with 128 bytes.
template <class P, bool YPASS>
struct ColStep {
    static constexpr int C = (YPASS && sizeof(typename P::S) == 8 ? 64 : 128) / (int)sizeof(typename P::S);
};

// one column (T = N/8 threads, thread j) of a tile; valid == false for the columns
// of the last tile beyond kx = N/2 (they compute on zeros and store nothing)
template <class Pin, class P, class Pout, int N, int SIGN, int CW, bool RF = false>
__device__ __forceinline__ void col_body(const typename Pin::S* src, typename Pout::S* dst, size_t base,
                                         size_t row_stride, bool valid, int j, ColSmem<P, CW>& csm,
                                         const typename P::S* __restrict__ tw) {
    typedef typename P::R R;
    constexpr int T = N / 8;
    cx<R> v[8];
#pragma unroll
    for (int s = 0; s < 8; s++) {
        if (valid) v[s] = Convert<Pin, P>::go(Pin::load(src[base + (size_t)(j + T * s) * row_stride]));
        else v[s] = cmake<R>(P::from_f64(0.0), P::from_f64(0.0));
    }
    fft<P, N, ColSmem<P, CW>, false, RF, false, false>(v, j, tw, 1, csm, SIGN);   // outputs go to W or FP64
    if (valid) {
#pragma unroll
        for (int s = 0; s < 8; s++) dst[base + (size_t)(j + T * s) * row_stride] = Pout::pack(Convert<P, Pout>::go(v[s]));
    }
}

// NC columns per plane: N/2 + 1 (half spectrum of a real field) or N (complex field)
template <class Pin, class P, class Pout, int N, int SIGN, int NC = N / 2 + 1, int CW = ColShape<P>::C>
__global__ void __launch_bounds__(CW * N / 8) k_col(const typename Pin::S* src, typename Pout::S* dst,
                                                               size_t plane_stride, size_t row_stride,
                                                               const typename P::S* __restrict__ tw) {
    constexpr int C = CW;
    extern __shared__ __align__(16) unsigned char smraw[];
    typename P::S* sm = reinterpret_cast<typename P::S*>(smraw);
    const int c = threadIdx.x % C, j = threadIdx.x / C;
    const int kx = blockIdx.x * C + c;
    ColSmem<P, C> csm{sm, c};
    tw = stage_table(tw, sm + N * C, N);
    col_body<Pin, P, Pout, N, SIGN, C>(src, dst, (size_t)blockIdx.y * plane_stride + kx, row_stride, kx < NC, j, csm, tw);
}

// inverse column FFT from an FP64 spectral array into W (precision P); the source is
// src1 when dev != NULL and dev->phase == 1, src0 otherwise (the current level's array)
template <class P, int N, int NC = N / 2 + 1, int CW = ColShape<P>::C>
__global__ void __launch_bounds__(CW * N / 8) k_col_sel(const double2* src0, const double2* src1,
                                                                   const KgDev* dev, typename P::S* dst,
                                                                   size_t plane_stride, size_t row_stride,
                                                                   const typename P::S* __restrict__ tw) {
    constexpr int C = CW;
    extern __shared__ __align__(16) unsigned char smraw[];
    typename P::S* sm = reinterpret_cast<typename P::S*>(smraw);
    const double2* src = (dev != nullptr && dev->phase) ? src1 : src0;
    const int c = threadIdx.x % C, j = threadIdx.x / C;
    const int kx = blockIdx.x * C + c;
    ColSmem<P, C> csm{sm, c};
    tw = stage_table(tw, sm + N * C, N);
    col_body<PrecF64, P, P, N, +1, C>(src, dst, (size_t)blockIdx.y * plane_stride + kx, row_stride, kx < NC, j, csm, tw);
}

// ---------------------------------------------------------------------------
// Fused z column: forward z FFT -> F^n, FP64 update, optional Q terms, inverse z FFT,
// in one pass over W (the batched ensemble's z pass; the single-state step runs the
// three parts as separate kernels, which measured faster at 512^3).
// coef[m2] = (2 c_k, 2 beta_k) for integer m2 = mx^2 + my^2 + mz^2; w2[m2] = omega_k^2.
// ---------------------------------------------------------------------------
// one (ky, kx) column (T = N/8 threads, thread j); update == false leaves the state
// untouched (a frozen instance); Q terms are added to q when want_q.
// PF: the state rows this thread updates are prefetched into shared memory by
// asynchronous copies issued before the forward FFT: 0 none, 1 uh^n only (st_sm holds
// 8 nt double2, slot s nt + tid), 2 both arrays (16 nt double2, uh^n at (2s) nt + tid,
// uh^{n-1} at (2s+1) nt + tid); nt = threads of the CTA, tid = this thread's slot.
template <class P, int N, int PF = 0, int CW = ColShape<P>::C, bool RF = false>
__device__ __forceinline__ void z_body(typename P::S* __restrict__ W, const double2* __restrict__ cur,
                                       double2* __restrict__ old, int kx, int ky, bool valid, int j,
                                       ColSmem<P, CW>& csm, const typename P::S* __restrict__ tw,
                                       const double2* __restrict__ coef, const double* __restrict__ w2tab,
                                       double inv_dt, bool update, bool want_q, NSum& q, double2* st_sm = nullptr,
                                       int tid = 0, int nt = 0) {
    typedef typename P::R R;
    typedef cx<R> Cx;
    constexpr int T = N / 8, NH = N / 2 + 1;
    const size_t rs = (size_t)N * NH;
    const size_t base = (size_t)ky * NH + kx;

    if (PF > 0 && valid) {
#pragma unroll
        for (int s = 0; s < 8; s++) {
            const size_t idx = base + (size_t)(j + T * s) * rs;
            cp_async16(st_sm + (size_t)(PF > 1 ? 2 * s : s) * nt + tid, cur + idx);
            if (PF > 1) cp_async16(st_sm + (size_t)(2 * s + 1) * nt + tid, old + idx);
        }
    }
    if (PF > 0) cp_async_commit();

    Cx v[8];
#pragma unroll
    for (int s = 0; s < 8; s++) {
        if (valid) v[s] = P::load(W[base + (size_t)(j + T * s) * rs]);
        else v[s] = cmake<R>(P::from_f64(0.0), P::from_f64(0.0));
    }
    // forward z transform, the update, then the inverse z transform; the double-float and
    // FP64 bodies are large, so they run both transforms through one copy of the FFT code
    constexpr bool kShare = sizeof(typename P::S) == 16;
#pragma unroll(kShare ? 1 : 2)
    for (int dir = 0; dir < 2; dir++) {
        fft<P, N, ColSmem<P, CW>, false, RF, false>(v, j, tw, 1, csm, dir == 0 ? -1 : +1);
        if (dir == 1) break;
        if (PF > 0) cp_async_wait_all();   // each thread reads back only its own copies
        const int my = ky <= N / 2 ? ky : ky - N;
        const int mxy2 = kx * kx + my * my;
        const double wgt = (kx == 0 || kx == N / 2) ? 1.0 : 2.0;
#pragma unroll
        for (int s = 0; s < 8; s++) {
            const int kz = j + T * s;
            const int mz = kz <= N / 2 ? kz : kz - N;
            const int m2 = mxy2 + mz * mz;
            if (valid) {
                const size_t idx = base + (size_t)kz * rs;
                const double2 cf = __ldg(coef + m2);
                const double2 a = PF > 0 ? st_sm[(size_t)(PF > 1 ? 2 * s : s) * nt + tid] : cur[idx];
                const double2 b = PF > 1 ? st_sm[(size_t)(2 * s + 1) * nt + tid] : old[idx];
                double nre = P::fma_into(cf.y, v[s].re, fma(cf.x, a.x, -b.x));
                double nim = P::fma_into(cf.y, v[s].im, fma(cf.x, a.y, -b.y));
                if (update) old[idx] = make_double2(nre, nim);
                if (want_q) {
                    const double dre = (nre - a.x) * inv_dt, dim = (nim - a.y) * inv_dt;
                    const double sre = nre + a.x, sim = nim + a.y;
                    const double term =
                        0.5 * (dre * dre + dim * dim) + 0.125 * __ldg(w2tab + m2) * (sre * sre + sim * sim);
                    q.add(wgt * term);
                }
                v[s] = cmake<R>(P::from_f64(nre), P::from_f64(nim));
            }
        }
    }
    if (valid) {
#pragma unroll
        for (int s = 0; s < 8; s++) W[base + (size_t)(j + T * s) * rs] = P::pack(v[s]);
    }
}

// ---------------------------------------------------------------------------
// Time-stepping schemes of the per-mode update.
// SCHEME 0, Eq. (2): cur = uh^n, old = uh^{n-1};
//     uh^{n+1} = 2 c_k uh^n - uh^{n-1} + 2 beta_k F^n_k   written over old.
// SCHEME 1, the fourth-order composition (triple jump) of Eq. (2) in kick-drift-kick
// form: cur = a (= uh), old = P (velocity variable); substep s = dev->sub of a step
//     P <- P + K_s (F - omega^2 a),   a <- a + h_s P       (both written back)
// with the merged kick K_s = (h_{s-1}/2)/(1 + omega^2 h_{s-1}^2/4) + (h_s/2)/(1 + omega^2
// h_s^2/4) (h_{-1} = h_2 = h_0) and h = (g1, g2, g1) dt.  One F per substep; with one
// substep of length dt this is Eq. (2) itself.
// ---------------------------------------------------------------------------
// (the tables and substep lengths travel in C4Args, kg_launch.h)

// The per-mode update of one step (or substep) at mode index idx with integer norm m2, F the
// transform of the cube there in the pass precision; writes the state (unless frozen) and
// returns the new uh in FP64, the value the inverse transforms start from.
template <class P, int SCHEME>
__device__ __forceinline__ double2 mode_update(cx<typename P::R> f, double2* cur, double2* old, size_t idx, int m2,
                                               const double2* __restrict__ coef, const C4Args& c4, int sub,
                                               bool update, double2 a) {
    const double2 b = old[idx];
    if constexpr (SCHEME == 0) {
        const double2 cf = __ldg(coef + m2);
        const double nre = P::fma_into(cf.y, f.re, fma(cf.x, a.x, -b.x));
        const double nim = P::fma_into(cf.y, f.im, fma(cf.x, a.y, -b.y));
        if (update) old[idx] = make_double2(nre, nim);
        return make_double2(nre, nim);
    } else {
        const double2 kc = __ldg(c4.kick + (size_t)sub * c4.stride + m2);
        const double pre = P::fma_into(kc.x, f.re, fma(-kc.y, a.x, b.x));
        const double pim = P::fma_into(kc.x, f.im, fma(-kc.y, a.y, b.y));
        const double2 n = make_double2(fma(c4.h[sub], pre, a.x), fma(c4.h[sub], pim, a.y));
        if (update) {
            old[idx] = make_double2(pre, pim);
            cur[idx] = n;
        }
        return n;
    }
}

// ---------------------------------------------------------------------------
// Streaming update between the forward and the inverse z FFT.  W holds F^n_k on entry
// and uh^{n+1}_k in the pass precision on exit; the state update and the Q terms are
// those of z_body.
// ---------------------------------------------------------------------------
// The mode stored at index i of a spectral array: the half spectrum of a real field
// ([kz][ky][kx], kx = 0..N/2) or the full spectrum of a complex field (kx = 0..N-1 in
// FFT order).  m2 = mx^2 + my^2 + mz^2 indexes the coefficient tables; w is the
// Parseval weight of the mode in the energy sums.
template <int N, bool CPLX>
struct ModeIndex {
    static constexpr int NX = CPLX ? N : N / 2 + 1;
    static constexpr long long kModes = (long long)N * N * NX;
    static_assert(kModes < (1ll << 31), "mode indexes fit 32 bits");
    int m2;
    bool twice;
    __device__ __forceinline__ explicit ModeIndex(unsigned i) {
        const unsigned row = i / NX;
        const int kx = (int)(i - row * NX);
        const int ky = (int)(row % N);
        const int kz = (int)(row / N);
        const int mx = (CPLX && kx > N / 2) ? kx - N : kx;
        const int my = ky <= N / 2 ? ky : ky - N, mz = kz <= N / 2 ? kz : kz - N;
        m2 = mx * mx + my * my + mz * mz;
        twice = !CPLX && kx != 0 && kx != N / 2;
    }
};

constexpr int kUpdThreads = 256;
constexpr int kSumThreads = 1024;   // second reduction stage of the update's Q partials

// One term of Q^{n+1/2} without its constant factor 1/(2 dt^2):
//     w_k ( |a1 - a0|^2 + r_k |a1 + a0|^2 ),   r_k = qr omega_k^2,  qr = dt^2 / 4,
// (the Q definition of kg.h multiplied by 2 dt^2).  Only the cancelling differences
// a1 - a0 are formed in FP64; the sums a1 + a0, r_k, the squares and their sums are
// formed in double-float on the FP32 pipe (the FP64 pipe already carries the update),
// except for the IEEE FP64 passes, which stay in FP64.
template <class P>
struct QTerm {
    typedef df T;
    static __device__ __forceinline__ T zero() { return df_make(0.f, 0.f); }
    // the cancelling differences in FP64, then squares and sums in double-float left
    // unnormalised: D, S and r S are sums of non-negative terms (n + a adds two values of
    // the same mode), so an unnormalised pair still holds each to within u^2 of its size,
    // and value() converts both words exactly
    static __device__ __forceinline__ T term(double n_re, double n_im, double2 a, double w2, double qr, bool twice) {
        const df dre = d2df_int(n_re - a.x), dim = d2df_int(n_im - a.y);
        const df sre = df_add_lazy(d2df_int(n_re), d2df_int(a.x)), sim = df_add_lazy(d2df_int(n_im), d2df_int(a.y));
        const df D = df_add_lazy(df_mul_lazy(dre, dre), df_mul_lazy(dim, dim));
        const df S = df_add_lazy(df_mul_lazy(sre, sre), df_mul_lazy(sim, sim));
        const df t = df_add_lazy(D, df_mul_lazy(df_mul_lazy(d2df_int(w2), d2df_int(qr)), S));
        return twice ? df_scale2(t, 2.0f) : t;
    }
    static __device__ __forceinline__ T add(T x, T y) { return df_add_lazy(x, y); }
    static __device__ __forceinline__ T shfl_down(T x, int o) {
        return df_make(__shfl_down_sync(0xffffffffu, x.hi, o), __shfl_down_sync(0xffffffffu, x.lo, o));
    }
    static __device__ __forceinline__ double value(T x) { return f2d_int(x.hi) + f2d_int(x.lo); }
};
template <>
struct QTerm<PrecF64> {
    typedef double T;
    static __device__ __forceinline__ T zero() { return 0.0; }
    static __device__ __forceinline__ T term(double n_re, double n_im, double2 a, double w2, double qr, bool twice) {
        const double r = qr * w2;
        const double dre = n_re - a.x, dim = n_im - a.y, sre = n_re + a.x, sim = n_im + a.y;
        const double t = fma(r, fma(sre, sre, sim * sim), fma(dre, dre, dim * dim));
        return twice ? t + t : t;
    }
    static __device__ __forceinline__ T add(T x, T y) { return x + y; }
    static __device__ __forceinline__ T shfl_down(T x, int o) { return __shfl_down_sync(0xffffffffu, x, o); }
    static __device__ __forceinline__ double value(T x) { return x; }
};

// pairwise (tree) sum of one value per thread of an NT-thread CTA; the total lands in
// thread 0
template <class Q, int NT>
__device__ __forceinline__ typename Q::T block_tree_sum(typename Q::T v, typename Q::T* sm) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = Q::add(v, Q::shfl_down(v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sm[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < NT / 32 ? sm[l] : Q::zero();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = Q::add(v, Q::shfl_down(v, o));
    }
    return v;
}

// Streaming per-mode update of Eq. (2) between the forward and the inverse z column
// passes, one mode per thread (a full grid keeps enough loads in flight to stream at
// HBM rate and lets the FP64 update overlap them):
//     uh^{n+1} = 2 c_k uh^n - uh^{n-1} + 2 beta_k F^n_k        (FP64, over uh^{n-1})
// and W <- uh^{n+1} in the pass precision for the inverse transforms.  On recording
// steps each CTA also writes its partial sum of the Q terms (QTerm) times qc = 1/(2 dt^2).
template <class P, int N, bool CPLX = false, int SCHEME = 0>
__global__ void __launch_bounds__(kUpdThreads, 6) k_update(typename P::S* __restrict__ W, double2* S0, double2* S1,
                                                          KgDev* __restrict__ dev, double* __restrict__ part_sum,
                                                          const double2* __restrict__ coef,
                                                          const double* __restrict__ w2tab, double qr, double qc,
                                                          C4Args c4) {
    typedef typename P::R R;
    typedef QTerm<P> Q;
    typedef ModeIndex<N, CPLX> MI;
    constexpr unsigned kModes = (unsigned)MI::kModes;
    static_assert(MI::kModes < (1ll << 31), "mode indexes fit 32 bits");
    __shared__ typename Q::T red[kUpdThreads / 32];
    const bool want_q = SCHEME == 0 && kg_recording(dev);
    const bool update = dev->frozen == 0;
    double2* __restrict__ cur = dev->phase ? S1 : S0;
    double2* __restrict__ old = dev->phase ? S0 : S1;
    const unsigned i = blockIdx.x * kUpdThreads + threadIdx.x;
    typename Q::T q = Q::zero();
    if (i < kModes) {
        const MI mi((unsigned)i);
        const cx<R> f = P::load(W[i]);
        const double2 a = cur[i];
        const double2 n = mode_update<P, SCHEME>(f, cur, old, i, mi.m2, coef, c4, dev->sub, update, a);
        W[i] = P::pack(cmake<R>(P::from_f64(n.x), P::from_f64(n.y)));
        if (want_q) q = Q::term(n.x, n.y, a, __ldg(w2tab + mi.m2), qr, mi.twice);
    }
    if (want_q) {
        q = block_tree_sum<Q, kUpdThreads>(q, red);
        if (threadIdx.x == 0) part_sum[blockIdx.x] = qc * Q::value(q);
    }
}

// ---------------------------------------------------------------------------
// z pass of the single-state step in one kernel: per (ky, kx) column, the forward z
// FFT -> F^n_k, the update of k_update (uh^{n+1} over uh^{n-1}, W <- uh^{n+1} in the pass
// precision, Q terms on recording steps), then the inverse z FFT of uh^{n+1}.  One pass
// over W: 2 W + 3 S per launch instead of 6 W + 3 S for the three kernels.  The state
// rows are read with plain loads after the forward transform (staging them in shared
// memory by cp.async before it cost more occupancy than it hid latency).
// C columns of N rows per CTA; C = 8 (128-byte double-float rows, 64-byte FP32 rows),
// 16 at N = 16 so that a CTA is at least one warp.
// ---------------------------------------------------------------------------
template <int N>
struct ZStepShape {
    static constexpr int C = N >= 32 ? 8 : 16;
    static constexpr int NT = C * N / 8;
};
// resident threads per SM the kernel is compiled for: 1024 (64 registers); 1536 for the
// FP32 passes at N = 512, whose smaller body fits 40 registers and gains from the extra
// loads in flight (1.046 -> 1.005 ms; not measured at other sizes, which keep 1024)
template <class P, int N>
struct ZStepMinBlocks {
    static constexpr int kThreads = (sizeof(typename P::S) == 8 && N >= 512) ? 1536 : 1024;
    static constexpr int value = kThreads / ZStepShape<N>::NT > 1 ? kThreads / ZStepShape<N>::NT : 1;
};

template <class P, int N, bool CPLX = false, int SCHEME = 0>
__global__ void __launch_bounds__(ZStepShape<N>::NT, ZStepMinBlocks<P, N>::value)
    k_zstep(typename P::S* __restrict__ W, double2* S0, double2* S1, KgDev* __restrict__ dev,
            double* __restrict__ part_sum, const typename P::S* __restrict__ tw, const double2* __restrict__ coef,
            const double* __restrict__ w2tab, double qr, double qc, C4Args c4) {
    typedef typename P::R R;
    typedef typename P::S S;
    typedef QTerm<P> Q;
    constexpr int T = N / 8, C = ZStepShape<N>::C, NT = ZStepShape<N>::NT;
    constexpr int NX = CPLX ? N : N / 2 + 1;   // columns per plane
    extern __shared__ __align__(16) unsigned char smraw[];
    S* sm = reinterpret_cast<S*>(smraw);
    __shared__ typename Q::T red[NT / 32];
    const int c = threadIdx.x % C, j = threadIdx.x / C;
    const int kx = blockIdx.x * C + c, ky = blockIdx.y;
    const bool valid = kx < NX;   // columns of the last tile beyond the plane compute on zeros
    ColSmem<P, C> csm{sm, c};
    tw = stage_table(tw, sm + N * C, N);
    const size_t rs = (size_t)N * NX, base = (size_t)ky * NX + kx;

    cx<R> v[8];
#pragma unroll
    for (int s = 0; s < 8; s++) {
        if (valid) v[s] = P::load(W[base + (size_t)(j + T * s) * rs]);
        else v[s] = cmake<R>(P::from_f64(0.0), P::from_f64(0.0));
    }
    typename Q::T q = Q::zero();
    // the 16-byte bodies are large: both transforms run through one copy of the FFT code
    constexpr bool kShare = sizeof(S) == 16;
#pragma unroll(kShare ? 1 : 2)
    for (int dir = 0; dir < 2; dir++) {
        // F^n goes to the update through exact conversions of both words, uh^{n+1} to W
        fft<P, N, ColSmem<P, C>, false, false, false>(v, j, tw, 1, csm, dir == 0 ? -1 : +1);
        if (dir == 1) break;
        // the run state is read only now, so that nothing of it is live across the
        // forward transform (at 64 registers: 132 -> 8 bytes of spills, 1.98 -> 1.91 ms
        // for the double-float pass at 512^3)
        const bool want_q = SCHEME == 0 && kg_recording(dev);
        const bool update = dev->frozen == 0;
        double2* __restrict__ cur = dev->phase ? S1 : S0;
        double2* __restrict__ old = dev->phase ? S0 : S1;
        const int mx = (CPLX && kx > N / 2) ? kx - N : kx;
        const int my = ky <= N / 2 ? ky : ky - N;
        const int mxy2 = mx * mx + my * my;
        const bool twice = !CPLX && kx != 0 && kx != N / 2;
        const int sub = SCHEME == 0 ? 0 : dev->sub;
#pragma unroll
        for (int s = 0; s < 8; s++) {
            const int kz = j + T * s;
            const int mz = kz <= N / 2 ? kz : kz - N;
            const int m2 = mxy2 + mz * mz;
            if (valid) {
                const size_t idx = base + (size_t)kz * rs;
                const double2 a = cur[idx];
                const double2 n = mode_update<P, SCHEME>(v[s], cur, old, idx, m2, coef, c4, sub, update, a);
                if (want_q) q = Q::add(q, Q::term(n.x, n.y, a, __ldg(w2tab + m2), qr, twice));
                v[s] = cmake<R>(P::from_f64(n.x), P::from_f64(n.y));
            }
        }
    }
    if (valid) {
#pragma unroll
        for (int s = 0; s < 8; s++) W[base + (size_t)(j + T * s) * rs] = P::pack(v[s]);
    }
    if (SCHEME == 0 && kg_recording(dev)) {
        q = block_tree_sum<Q, NT>(q, red);
        if (threadIdx.x == 0) part_sum[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = qc * Q::value(q);
    }
}

// second stage of the Q sum on recording steps: CTA b sums in[b*1024 ...] pairwise into out[b]
__global__ void __launch_bounds__(kSumThreads) k_sum_parts(const double* __restrict__ in, int count,
                                                           double* __restrict__ out, const KgDev* __restrict__ dev);

// ---------------------------------------------------------------------------
// finalisers (one CTA of 1024 threads)
// ---------------------------------------------------------------------------
constexpr int kFinThreads = 1024;

__device__ __forceinline__ void fin_reduce(const double* part_sum, const double* part_max, int count, NSum& acc,
                                           double& mx) {
    __shared__ double red[96];
    __shared__ unsigned long long kred[kFinThreads / 32];
    acc.s = 0.0;
    acc.c = 0.0;
    unsigned long long key = 0ull;
    for (int i = threadIdx.x; i < count; i += kFinThreads) {
        if (part_sum) acc.add(part_sum[i]);
        if (part_max) {
            const unsigned long long k = (unsigned long long)__double_as_longlong(part_max[i]);
            key = k > key ? k : key;
        }
    }
    if (part_max) key = block_max_key<kFinThreads>(key, kred);
    mx = __longlong_as_double((long long)key);
    if (part_sum) {
        double unused = 0.0;
        block_reduce<kFinThreads>(acc, unused, red);
    }
}

#ifdef KG_DEFINE_COMMON_KERNELS   // defined by exactly one translation unit
// after a stepping x pass: blow-up check and P^l; p_norm = lam h^3 / 4
__global__ void __launch_bounds__(kFinThreads) k_fin_x(const double* part_sum, const double* part_max, int count,
                                                       KgDev* dev, double p_norm) {
    NSum acc;
    double mx;
    // record_p marks the next step's x pass run ahead by kg_energy: it records P^l, and its
    // max |u| waits in maxabs_peek until that step runs (kg_status reports the last step's)
    const bool ahead = dev->record_p != 0;   // read by every thread before fin_reduce's barriers
    const bool rec = kg_recording(dev) || ahead;
    fin_reduce(rec ? part_sum : nullptr, part_max, count, acc, mx);
    if (dev->complex_field) mx = sqrt(mx);   // the keys were |u|^2
    // the composed scheme checks the field at integer times only (its first substep)
    if (threadIdx.x == 0 && dev->sub == 0) {
        if (!dev->frozen) {
            if (ahead) dev->maxabs_peek = mx;
            else dev->maxabs_last = mx;
            if (rec) {
                dev->P_last = p_norm * acc.value();
                dev->P_last_level = dev->level;
            }
            if (dev->threshold > 0.0 && !(mx <= dev->threshold)) {
                dev->frozen = 1;
                dev->blowup_level = dev->level;
            }
        }
    }
    if (threadIdx.x == 0) dev->record_p = 0;
}

// after a peek x pass
__global__ void __launch_bounds__(kFinThreads) k_fin_peek(const double* part_sum, const double* part_max, int count,
                                                          KgDev* dev, double p_norm) {
    NSum acc;
    double mx;
    fin_reduce(part_sum, part_max, count, acc, mx);
    if (dev->complex_field) mx = sqrt(mx);
    if (threadIdx.x == 0) {
        dev->P_peek = p_norm * acc.value();
        dev->maxabs_peek = mx;
    }
}

// after the update: Q^{l+1/2} (q_norm = h^3/N^3) and the level advance
__global__ void __launch_bounds__(kSumThreads) k_sum_parts(const double* __restrict__ in, int count,
                                                           double* __restrict__ out, const KgDev* __restrict__ dev) {
    if (!kg_recording(dev)) return;
    __shared__ double red[kSumThreads / 32];
    const int i = blockIdx.x * kSumThreads + threadIdx.x;
    double v = block_tree_sum<QTerm<PrecF64>, kSumThreads>(i < count ? in[i] : 0.0, red);
    if (threadIdx.x == 0) out[blockIdx.x] = v;
}

__global__ void __launch_bounds__(kFinThreads) k_fin_z(const double* part_sum, int count, KgDev* dev, double q_norm) {
    const bool rec = kg_recording(dev);
    NSum acc;
    double mx;
    if (rec) fin_reduce(part_sum, nullptr, count, acc, mx);
    if (threadIdx.x == 0 && !dev->frozen) {
        if (rec) {
            dev->Q_last = q_norm * acc.value();
            dev->Q_last_level = dev->level;
        }
        if (dev->scheme == 0) {
            dev->level += 1;
            dev->phase ^= 1;
        } else {   // composed scheme: the state arrays stay put; a step is three substeps
            dev->sub = dev->sub == 2 ? 0 : dev->sub + 1;
            if (dev->sub == 0) dev->level += 1;
        }
    }
}

#endif  // KG_DEFINE_COMMON_KERNELS

// ---------------------------------------------------------------------------
// FP64 set-up and read-out kernels
// ---------------------------------------------------------------------------
// forward R2C along x of physical lines: out[line][k] = sum_x f(u[line][x]) e^{-2 pi i k x/N},
// f(u) = u (cube == 0) or lam u^3 (cube == 1).  Same line mapping as pass X.
template <int N>
__global__ void __launch_bounds__(kXThreads) k_x_forward(const double* __restrict__ u, double2* __restrict__ out,
                                                         const double2* __restrict__ tw, int cube, double lam) {
    typedef PrecF64 P;
    typedef cx<double> C;
    typedef XShape<N> X;
    constexpr int M = X::M, T = X::T, NH = N / 2 + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    double2* sm = reinterpret_cast<double2*>(smraw);
    const int li = threadIdx.x / T, j = threadIdx.x % T;
    const size_t line = (size_t)blockIdx.x * X::LPC + li;
    const double* __restrict__ ul = u + line * N;
    double2* __restrict__ L = out + line * NH;
    LineSmem<P> lsm{sm + li * X::PADM};
    C v[8];
#pragma unroll
    for (int s = 0; s < 8; s++) {
        const int m = j + T * s;
        double a = ul[2 * m], b = ul[2 * m + 1];
        if (cube) {
            a = lam * (a * a * a);
            b = lam * (b * b * b);
        }
        v[s] = cmake<double>(a, b);
    }
    fft<P, M>(v, j, tw, 2, lsm, -1);
#pragma unroll
    for (int s = 0; s < 8; s++) lsm.put(j + T * s, v[s]);
    lsm.sync();
#pragma unroll
    for (int s = 0; s < 8; s++) {
        const int k = j + T * s;
        C Z = v[s];
        C Zp = lsm.get((M - k) & (M - 1));
        C A = Z + conj(Zp);
        C B = Z - conj(Zp);
        C w = twiddle<P>(tw, k, -1);
        C D = mul_i(cmul(w, B));
        L[k] = make_double2(0.5 * (A.re - D.re), 0.5 * (A.im - D.im));
        if (k == 0) L[M] = make_double2(Z.re - Z.im, 0.0);
    }
}

// inverse C2R along x to physical lines, times scale; optionally sum u^4 (per CTA)
template <int N>
__global__ void __launch_bounds__(kXThreads) k_x_inverse(const double2* __restrict__ in, double* __restrict__ u,
                                                         const double2* __restrict__ tw, double scale,
                                                         double* __restrict__ part_sum) {
    typedef PrecF64 P;
    typedef cx<double> C;
    typedef XShape<N> X;
    constexpr int M = X::M, T = X::T, NH = N / 2 + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    double2* sm = reinterpret_cast<double2*>(smraw);
    __shared__ double red[96];
    const int li = threadIdx.x / T, j = threadIdx.x % T;
    const size_t line = (size_t)blockIdx.x * X::LPC + li;
    LineSmem<P> lsm{sm + li * X::PADM};
    C v[8];
    x_load_c2r<P, N>(in + line * NH, j, tw, v);
    fft<P, M>(v, j, tw, 2, lsm, +1);
    NSum acc;
    acc.s = 0.0;
    acc.c = 0.0;
#pragma unroll
    for (int s = 0; s < 8; s++) {
        const int m = j + T * s;
        const double a = v[s].re * scale, b = v[s].im * scale;
        if (u) {
            u[line * N + 2 * m] = a;
            u[line * N + 2 * m + 1] = b;
        }
        if (part_sum) {
            const double a2 = a * a, b2 = b * b;
            acc.add(a2 * a2);
            acc.add(b2 * b2);
        }
    }
    if (part_sum) {
        double mx = 0.0;
        block_reduce<kXThreads>(acc, mx, red);
        if (threadIdx.x == 0) part_sum[blockIdx.x] = acc.value();
    }
}

// Set-up and read-out along x in the pass precision, two physical x-lines per N-point
// complex transform (the pair form of the x pass), one pair per N/8 threads:
// FWD: physical FP64 lines u_in (lam u^3 when cube) -> their half spectra, unnormalised,
//      in the pass precision in spec (lines of N/2 + 1);
// else: half spectra in spec -> physical lines times scale, FP64, into u_out.
template <class P, int N, bool FWD>
__global__ void __launch_bounds__(kXThreads) k_x_pair_io(const double* __restrict__ u_in, typename P::S* __restrict__ spec,
                                                         double* __restrict__ u_out,
                                                         const typename P::S* __restrict__ tw, int cube, double lam,
                                                         double scale) {
    typedef typename P::R R;
    typedef cx<R> C;
    typedef XpShape<N> X;
    constexpr int NH = N / 2 + 1, T = X::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    typename P::S* sm = reinterpret_cast<typename P::S*>(smraw);
    const int pi = threadIdx.x / T, j = threadIdx.x % T;
    const size_t pair = (size_t)blockIdx.x * X::PPC + pi;
    LineSmemX<P, X::CTA_SYNC> lsm{sm + pi * X::PADN, 1u + (unsigned)pi, (unsigned)T};
    typename P::S* __restrict__ L1 = spec + 2 * pair * NH;
    typename P::S* __restrict__ L2 = L1 + NH;
    C v[8];
    if constexpr (FWD) {
        const double* __restrict__ u1 = u_in + 2 * pair * N;
        const double* __restrict__ u2 = u1 + N;
        const R rlam = P::from_f64(lam);
#pragma unroll
        for (int s = 0; s < 8; s++) {
            const int x = j + T * s;
            R a = P::from_f64(u1[x]), b = P::from_f64(u2[x]);
            if (cube) {
                a = rlam * (a * a * a);
                b = rlam * (b * b * b);
            }
            v[s] = cmake<R>(a, b);
        }
        fft<P, N>(v, j, tw, 1, lsm, -1);
        x_pair_unpack<P, N>(L1, L2, j, lsm, v);
    } else {
        x_pair_load<P, N>(L1, L2, j, v);
        fft<P, N>(v, j, tw, 1, lsm, +1);
        double* __restrict__ o1 = u_out + 2 * pair * N;
        double* __restrict__ o2 = o1 + N;
#pragma unroll
        for (int s = 0; s < 8; s++) {
            const int x = j + T * s;
            const cx<double> w = Convert<P, PrecF64>::go(
                cmake<R>(P::scale2(v[s].re, scale), P::scale2(v[s].im, scale)));
            o1[x] = w.re;
            o2[x] = w.im;
        }
    }
}

// uh^{-1} = c_k uh^0 - dt vh^0 + beta_k F^0 (coef holds 2c, 2 beta); b holds vh^0 on entry
template <int N, bool CPLX = false>
__global__ void k_startup(const double2* __restrict__ a, double2* __restrict__ b, const double2* __restrict__ f,
                          const double2* __restrict__ coef, double dt) {
    typedef ModeIndex<N, CPLX> MI;
    const size_t total = (size_t)MI::kModes;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const double2 cf = coef[MI((unsigned)i).m2];
        const double c = 0.5 * cf.x, beta = 0.5 * cf.y;
        const double2 a0 = a[i], v0 = b[i], f0 = f[i];
        b[i] = make_double2(c * a0.x - dt * v0.x + beta * f0.x, c * a0.y - dt * v0.y + beta * f0.y);
    }
}

// startup of the composed scheme: b holds vh^0 on entry and the stored velocity variable
// P^0 = vh^0 - (h_0/2)(F^0 - omega^2 uh^0)/(1 + omega^2 h_0^2/4) on exit (the first
// merged kick then applies only the opening half kick); kick0 = (K_0, K_0 omega^2) with
// K_0 = h_0/(1 + omega^2 h_0^2/4)
template <int N>
__global__ void k_startup_c4(const double2* __restrict__ a, double2* __restrict__ b, const double2* __restrict__ f,
                             const double2* __restrict__ kick0) {
    typedef ModeIndex<N, false> MI;
    const size_t total = (size_t)MI::kModes;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const double2 kc = kick0[MI((unsigned)i).m2];
        const double2 a0 = a[i], v0 = b[i], f0 = f[i];
        b[i] = make_double2(v0.x - 0.5 * (kc.x * f0.x - kc.y * a0.x), v0.y - 0.5 * (kc.x * f0.y - kc.y * a0.y));
    }
}

// Q(x, y) partials for arbitrary FP64 spectral pairs (energy outside the recorded steps)
template <int N, bool CPLX = false>
__global__ void __launch_bounds__(256) k_energy_q(const double2* __restrict__ x, const double2* __restrict__ y,
                                                  const double* __restrict__ w2tab, double inv_dt,
                                                  double* __restrict__ part_sum) {
    typedef ModeIndex<N, CPLX> MI;
    __shared__ double red[96];
    const size_t total = (size_t)MI::kModes;
    NSum acc;
    acc.s = 0.0;
    acc.c = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const MI mi((unsigned)i);
        const double w = mi.twice ? 2.0 : 1.0;
        const double2 a = x[i], b = y[i];
        const double dre = (a.x - b.x) * inv_dt, dim = (a.y - b.y) * inv_dt;
        const double sre = a.x + b.x, sim = a.y + b.y;
        acc.add(w * (0.5 * (dre * dre + dim * dim) + 0.125 * w2tab[mi.m2] * (sre * sre + sim * sim)));
    }
    double mx = 0.0;
    block_reduce<256>(acc, mx, red);
    if (threadIdx.x == 0) part_sum[blockIdx.x] = acc.value();
}

#ifdef KG_DEFINE_COMMON_KERNELS
// plain Neumaier total of partials into *out (times norm)
__global__ void __launch_bounds__(kFinThreads) k_fin_sum(const double* part_sum, int count, double norm, double* out) {
    NSum acc;
    double mx;
    fin_reduce(part_sum, nullptr, count, acc, mx);
    if (threadIdx.x == 0) *out = norm * acc.value();
}

#endif  // KG_DEFINE_COMMON_KERNELS

}  // namespace kg
