// kg_launch_impl.cuh -- template launchers, instantiated once per precision.
#pragma once
#include <type_traits>
#include "kg_complex.cuh"
#include "kg_ensemble.cuh"
#include "kg_kernels.cuh"
#include "kg_launch.h"
#include "kg_xyfuse.cuh"

namespace kg {

// CTAs per cluster of the fused xy pass: a plane of FP32 W is 1.05 MB at N = 512, which
// eight CTAs hold in 136 KB of shared memory each
constexpr int kXyCluster = 8;

// dynamic shared memory limit of a kernel (static shared memory comes on top, so the
// attribute is set whatever the size)
template <class K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define KG_DISPATCH_N(N, ...)                               \
    switch (N) {                                            \
        case 16: { constexpr int NN = 16; __VA_ARGS__; }    \
        case 32: { constexpr int NN = 32; __VA_ARGS__; }    \
        case 64: { constexpr int NN = 64; __VA_ARGS__; }    \
        case 128: { constexpr int NN = 128; __VA_ARGS__; }  \
        case 256: { constexpr int NN = 256; __VA_ARGS__; }  \
        case 512: { constexpr int NN = 512; __VA_ARGS__; }  \
        default: return cudaErrorInvalidValue;              \
    }

template <class P>
struct Launchers {
    typedef typename P::S S;

    // persistent x pass: as many CTAs as fit on the device at once (both modes), at most
    // one per batch; cached per grid size
    template <int N>
    static size_t x_smem() {
        typedef XShape<N> X;
        return (size_t)(XPipelined<P>::value ? 2 : 1) * X::LPC * X::PADM * sizeof(S);
    }
    template <int N>
    static int x_grid_n() {
        static int grid = 0;
        if (!XPipelined<P>::value) return N * N / XShape<N>::LPC;
        if (grid == 0) {
            typedef XShape<N> X;
            int dev = 0, sms = 0, occ0 = 0, occ1 = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return 0;
            if (set_smem(k_pass_x<P, N, MODE_STEP>, x_smem<N>()) != cudaSuccess ||
                set_smem(k_pass_x<P, N, MODE_PEEK>, x_smem<N>()) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ0, k_pass_x<P, N, MODE_STEP>, kXThreads,
                                                              x_smem<N>()) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, k_pass_x<P, N, MODE_PEEK>, kXThreads,
                                                              x_smem<N>()) != cudaSuccess)
                return 0;
            const int occ = occ0 < occ1 ? occ0 : occ1;
            const int nb = N * N / X::LPC;
            grid = occ * sms < nb ? occ * sms : nb;
            if (grid < 1) grid = 1;
        }
        return grid;
    }
    template <int N>
    static cudaError_t pass_x_n(int mode, void* W, KgDev* dev, double* ps, double* pm, const void* tw, double scale,
                                double lam, cudaStream_t st) {
        const size_t smem = x_smem<N>();
        const int grid = x_grid_n<N>();
        if (grid == 0) return cudaErrorInvalidConfiguration;
        if (mode == MODE_STEP) {
            cudaError_t e = set_smem(k_pass_x<P, N, MODE_STEP>, smem);
            if (e != cudaSuccess) return e;
            k_pass_x<P, N, MODE_STEP><<<grid, kXThreads, smem, st>>>((S*)W, dev, ps, pm, (const S*)tw, scale, lam);
        } else {
            cudaError_t e = set_smem(k_pass_x<P, N, MODE_PEEK>, smem);
            if (e != cudaSuccess) return e;
            k_pass_x<P, N, MODE_PEEK><<<grid, kXThreads, smem, st>>>((S*)W, dev, ps, pm, (const S*)tw, scale, lam);
        }
        return cudaGetLastError();
    }
    static cudaError_t pass_x(int N, int mode, void* W, KgDev* dev, double* ps, double* pm, const void* tw,
                              double scale, double lam, cudaStream_t st) {
        KG_DISPATCH_N(N, return pass_x_n<NN>(mode, W, dev, ps, pm, tw, scale, lam, st));
    }
    // partials the x pass writes (its grid); 0 when the device cannot be queried
    static int x_parts(int N) {
        KG_DISPATCH_N(N, return x_grid_n<NN>());
    }

    template <int N, int SIGN, int NC = N / 2 + 1, int C = ColShape<P>::C>
    static cudaError_t col_n(void* W, size_t pstride, size_t rstride, int nplanes, const void* tw, cudaStream_t st) {
        const size_t smem = (size_t)(N * C + N) * sizeof(S);
        auto kern = k_col<P, P, P, N, SIGN, NC, C>;
        cudaError_t e = set_smem(kern, smem);
        if (e != cudaSuccess) return e;
        dim3 grid((NC + C - 1) / C, nplanes);
        kern<<<grid, C * N / 8, smem, st>>>((const S*)W, (S*)W, pstride, rstride, (const S*)tw);
        return cudaGetLastError();
    }
    // y passes (row stride of one x-row) and z passes (row stride of a plane) take the
    // tile widths of ColStep
    template <int N, int SIGN, int NC>
    static cudaError_t col_yz(void* W, size_t pstride, size_t rstride, int nplanes, const void* tw,
                              cudaStream_t st) {
        if (rstride <= (size_t)N)
            return col_n<N, SIGN, NC, ColStep<P, true>::C>(W, pstride, rstride, nplanes, tw, st);
        return col_n<N, SIGN, NC, ColStep<P, false>::C>(W, pstride, rstride, nplanes, tw, st);
    }
    static cudaError_t col(int N, int sign, void* W, size_t pstride, size_t rstride, int nplanes, const void* tw,
                           cudaStream_t st) {
        if (sign < 0) { KG_DISPATCH_N(N, return (col_yz<NN, -1, NN / 2 + 1>(W, pstride, rstride, nplanes, tw, st))); }
        KG_DISPATCH_N(N, return (col_yz<NN, +1, NN / 2 + 1>(W, pstride, rstride, nplanes, tw, st)));
    }

    template <int N, int NC = N / 2 + 1>
    static cudaError_t col_from_f64_n(const double2* src0, const double2* src1, const KgDev* dev, void* W,
                                      size_t pstride, size_t rstride, int nplanes, const void* tw, cudaStream_t st) {
        constexpr int C = ColShape<P>::C;
        const size_t smem = (size_t)(N * C + N) * sizeof(S);
        auto kern = k_col_sel<P, N, NC, C>;
        cudaError_t e = set_smem(kern, smem);
        if (e != cudaSuccess) return e;
        dim3 grid((NC + C - 1) / C, nplanes);
        kern<<<grid, C * N / 8, smem, st>>>(src0, src1, dev, (S*)W, pstride, rstride, (const S*)tw);
        return cudaGetLastError();
    }
    static cudaError_t col_from_f64(int N, const double2* src0, const double2* src1, const KgDev* dev, void* W,
                                    size_t pstride, size_t rstride, int nplanes, const void* tw, cudaStream_t st) {
        KG_DISPATCH_N(N, return col_from_f64_n<NN>(src0, src1, dev, W, pstride, rstride, nplanes, tw, st));
    }

    // set-up and read-out transforms in the pass precision (double-float only: the FP32
    // passes would degrade the FP64 state, and the FP64 passes have their own kernels)
    static constexpr bool kPassIO = std::is_same<P, PrecDF>::value;
    template <int N, bool FWD>
    static cudaError_t x_io_n(const double* u_in, void* spec, double* u_out, const void* tw, int cube, double lam,
                              double scale, cudaStream_t st) {
        typedef XpShape<N> X;
        const size_t smem = (size_t)X::PPC * X::PADN * sizeof(S);
        auto kern = k_x_pair_io<P, N, FWD>;
        cudaError_t e = set_smem(kern, smem);
        if (e != cudaSuccess) return e;
        kern<<<N * N / 2 / X::PPC, kXThreads, smem, st>>>(u_in, (S*)spec, u_out, (const S*)tw, cube, lam, scale);
        return cudaGetLastError();
    }
    static cudaError_t x_setup(int N, const double* u, void* spec, const void* tw, int cube, double lam,
                               cudaStream_t st) {
        if constexpr (!kPassIO) return cudaErrorNotSupported;
        else { KG_DISPATCH_N(N, return (x_io_n<NN, true>(u, spec, nullptr, tw, cube, lam, 1.0, st))); }
    }
    static cudaError_t x_readout(int N, void* spec, double* u, const void* tw, double scale, cudaStream_t st) {
        if constexpr (!kPassIO) return cudaErrorNotSupported;
        else { KG_DISPATCH_N(N, return (x_io_n<NN, false>(nullptr, spec, u, tw, 0, 0.0, scale, st))); }
    }
    // forward column FFT from W (pass precision) into an FP64 spectral array
    template <int N>
    static cudaError_t col_to_f64_n(const void* W, double2* out, size_t pstride, size_t rstride, int nplanes,
                                    const void* tw, cudaStream_t st) {
        constexpr int C = ColShape<P>::C, NH = N / 2 + 1;
        const size_t smem = (size_t)(N * C + N) * sizeof(S);
        auto kern = k_col<P, P, PrecF64, N, -1, NH, C>;
        cudaError_t e = set_smem(kern, smem);
        if (e != cudaSuccess) return e;
        dim3 grid((NH + C - 1) / C, nplanes);
        kern<<<grid, C * N / 8, smem, st>>>((const S*)W, out, pstride, rstride, (const S*)tw);
        return cudaGetLastError();
    }
    static cudaError_t col_to_f64(int N, const void* W, double2* out, size_t pstride, size_t rstride, int nplanes,
                                  const void* tw, cudaStream_t st) {
        if constexpr (!kPassIO) return cudaErrorNotSupported;
        else { KG_DISPATCH_N(N, return (col_to_f64_n<NN>(W, out, pstride, rstride, nplanes, tw, st))); }
    }

    // the same for a complex field (one N-point transform per line, N columns per plane)
    template <int N, bool FWD>
    static cudaError_t xc_io_n(const double2* u_in, void* spec, double2* u_out, const void* tw, int cube,
                               double lam, double scale, cudaStream_t st) {
        typedef XcShape<N> X;
        const size_t smem = (size_t)X::LPC * X::PADN * sizeof(S);
        auto kern = k_xc_io<P, N, FWD>;
        cudaError_t e = set_smem(kern, smem);
        if (e != cudaSuccess) return e;
        kern<<<N * N / X::LPC, kXThreads, smem, st>>>(u_in, (S*)spec, u_out, (const S*)tw, cube, lam, scale);
        return cudaGetLastError();
    }
    static cudaError_t xc_setup(int N, const double2* u, void* spec, const void* tw, int cube, double lam,
                                cudaStream_t st) {
        if constexpr (!kPassIO) return cudaErrorNotSupported;
        else { KG_DISPATCH_N(N, return (xc_io_n<NN, true>(u, spec, nullptr, tw, cube, lam, 1.0, st))); }
    }
    static cudaError_t xc_readout(int N, void* spec, double2* u, const void* tw, double scale, cudaStream_t st) {
        if constexpr (!kPassIO) return cudaErrorNotSupported;
        else { KG_DISPATCH_N(N, return (xc_io_n<NN, false>(nullptr, spec, u, tw, 0, 0.0, scale, st))); }
    }
    template <int N>
    static cudaError_t colc_to_f64_n(const void* W, double2* out, size_t pstride, size_t rstride, int nplanes,
                                     const void* tw, cudaStream_t st) {
        constexpr int C = ColShape<P>::C;
        const size_t smem = (size_t)(N * C + N) * sizeof(S);
        auto kern = k_col<P, P, PrecF64, N, -1, N, C>;
        cudaError_t e = set_smem(kern, smem);
        if (e != cudaSuccess) return e;
        dim3 grid((N + C - 1) / C, nplanes);
        kern<<<grid, C * N / 8, smem, st>>>((const S*)W, out, pstride, rstride, (const S*)tw);
        return cudaGetLastError();
    }
    static cudaError_t colc_to_f64(int N, const void* W, double2* out, size_t pstride, size_t rstride, int nplanes,
                                   const void* tw, cudaStream_t st) {
        if constexpr (!kPassIO) return cudaErrorNotSupported;
        else { KG_DISPATCH_N(N, return (colc_to_f64_n<NN>(W, out, pstride, rstride, nplanes, tw, st))); }
    }

    static int update_parts(int N) { return (int)(((long long)N * N * (N / 2 + 1) + kUpdThreads - 1) / kUpdThreads); }
    template <int N>
    static cudaError_t update_n(void* W, double2* S0, double2* S1, KgDev* dev, double* ps, const double2* coef,
                                const double* w2, double inv_dt, const C4Args* c4, cudaStream_t st) {
        const double qr = 0.25 / (inv_dt * inv_dt), qc = 0.5 * inv_dt * inv_dt;
        if (c4) {
            k_update<P, N, false, 1><<<update_parts(N), kUpdThreads, 0, st>>>((S*)W, S0, S1, dev, ps, coef, w2, qr,
                                                                              qc, *c4);
        } else {
            k_update<P, N><<<update_parts(N), kUpdThreads, 0, st>>>((S*)W, S0, S1, dev, ps, coef, w2, qr, qc,
                                                                   C4Args{});
        }
        return cudaGetLastError();
    }
    static cudaError_t update(int N, void* W, double2* S0, double2* S1, KgDev* dev, double* ps, const double2* coef,
                              const double* w2, double inv_dt, const C4Args* c4, cudaStream_t st) {
        KG_DISPATCH_N(N, return update_n<NN>(W, S0, S1, dev, ps, coef, w2, inv_dt, c4, st));
    }
    // ---- complex field ----
    template <int N>
    static cudaError_t passc_x_n(int mode, void* W, KgDev* dev, double* ps, double* pm, const void* tw,
                                 double scale, double lam, cudaStream_t st) {
        typedef XcShape<N> X;
        const size_t smem = (size_t)X::LPC * X::PADN * sizeof(S);
        const int grid = N * N / X::LPC;
        if (mode == MODE_STEP) {
            cudaError_t e = set_smem(k_pass_xc<P, N, MODE_STEP>, smem);
            if (e != cudaSuccess) return e;
            k_pass_xc<P, N, MODE_STEP><<<grid, kXThreads, smem, st>>>((S*)W, dev, ps, pm, (const S*)tw, scale, lam);
        } else {
            cudaError_t e = set_smem(k_pass_xc<P, N, MODE_PEEK>, smem);
            if (e != cudaSuccess) return e;
            k_pass_xc<P, N, MODE_PEEK><<<grid, kXThreads, smem, st>>>((S*)W, dev, ps, pm, (const S*)tw, scale, lam);
        }
        return cudaGetLastError();
    }
    static cudaError_t passc_x(int N, int mode, void* W, KgDev* dev, double* ps, double* pm, const void* tw,
                               double scale, double lam, cudaStream_t st) {
        KG_DISPATCH_N(N, return passc_x_n<NN>(mode, W, dev, ps, pm, tw, scale, lam, st));
    }
    static int xc_parts(int N) { return N * N / (kXThreads / (N / 8)); }
    static cudaError_t colc(int N, int sign, void* W, size_t pstride, size_t rstride, int nplanes, const void* tw,
                            cudaStream_t st) {
        if (sign < 0) { KG_DISPATCH_N(N, return (col_yz<NN, -1, NN>(W, pstride, rstride, nplanes, tw, st))); }
        KG_DISPATCH_N(N, return (col_yz<NN, +1, NN>(W, pstride, rstride, nplanes, tw, st)));
    }
    static cudaError_t colc_from_f64(int N, const double2* src0, const double2* src1, const KgDev* dev, void* W,
                                     size_t pstride, size_t rstride, int nplanes, const void* tw, cudaStream_t st) {
        KG_DISPATCH_N(N, return (col_from_f64_n<NN, NN>(src0, src1, dev, W, pstride, rstride, nplanes, tw, st)));
    }
    static int updatec_parts(int N) { return (int)(((long long)N * N * N + kUpdThreads - 1) / kUpdThreads); }
    static cudaError_t updatec(int N, void* W, double2* S0, double2* S1, KgDev* dev, double* ps, const double2* coef,
                               const double* w2, double inv_dt, cudaStream_t st) {
        const double qr = 0.25 / (inv_dt * inv_dt), qc = 0.5 * inv_dt * inv_dt;
        KG_DISPATCH_N(N, {
            k_update<P, NN, true><<<updatec_parts(NN), kUpdThreads, 0, st>>>((S*)W, S0, S1, dev, ps, coef, w2, qr,
                                                                             qc, C4Args{});
            return cudaGetLastError();
        });
    }

    // fused z pass (forward z FFT, update, inverse z FFT) of a real (cplx = false) or
    // complex field, Eq. (2) (SCHEME 0) or the composed scheme (SCHEME 1, real field);
    // zstep_parts: the Q partials it writes when recording
    template <int N, bool CPLX, int SCHEME>
    static cudaError_t zstep_n(void* W, double2* S0, double2* S1, KgDev* dev, double* ps, const void* tw,
                               const double2* coef, const double* w2, double inv_dt, const C4Args& c4,
                               cudaStream_t st) {
        typedef ZStepShape<N> Z;
        constexpr int NX = CPLX ? N : N / 2 + 1;
        const size_t smem = (size_t)(N * Z::C + N) * sizeof(S);
        auto kern = k_zstep<P, N, CPLX, SCHEME>;
        cudaError_t e = set_smem(kern, smem);
        if (e != cudaSuccess) return e;
        const double qr = 0.25 / (inv_dt * inv_dt), qc = 0.5 * inv_dt * inv_dt;
        dim3 grid((NX + Z::C - 1) / Z::C, N);
        kern<<<grid, Z::NT, smem, st>>>((S*)W, S0, S1, dev, ps, (const S*)tw, coef, w2, qr, qc, c4);
        return cudaGetLastError();
    }
    static cudaError_t zstep(int N, bool cplx, void* W, double2* S0, double2* S1, KgDev* dev, double* ps,
                             const void* tw, const double2* coef, const double* w2, double inv_dt, const C4Args* c4,
                             cudaStream_t st) {
        if (cplx) {
            if (c4) return cudaErrorInvalidValue;   // the composed scheme is built for real fields
            KG_DISPATCH_N(N, return (zstep_n<NN, true, 0>(W, S0, S1, dev, ps, tw, coef, w2, inv_dt, C4Args{}, st)));
        }
        if (c4) { KG_DISPATCH_N(N, return (zstep_n<NN, false, 1>(W, S0, S1, dev, ps, tw, coef, w2, inv_dt, *c4, st))); }
        KG_DISPATCH_N(N, return (zstep_n<NN, false, 0>(W, S0, S1, dev, ps, tw, coef, w2, inv_dt, C4Args{}, st)));
    }
    static int zstep_parts(int N, bool cplx) {
        const int C = N >= 32 ? ZStepShape<32>::C : ZStepShape<16>::C;
        const int nx = cplx ? N : N / 2 + 1;
        return (nx + C - 1) / C * N;
    }

    // ---- fused inverse y / x / forward y pass (FP32 work array, real field) ----
    template <int N, bool DO_YI>
    static cudaLaunchConfig_t xy_config(cudaLaunchAttribute* attr, int grid, cudaStream_t st) {
        typedef XyShape<N, kXyCluster> X;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(X::NT);
        cfg.dynamicSmemBytes = (size_t)(X::SLAB + X::XBUF) * sizeof(float2);
        cfg.stream = st;
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kXyCluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cfg;
    }
    // persistent grid: as many clusters as fit on the device at once, at most one per
    // plane; cached per grid size (both variants share it)
    template <int N>
    static int xy_grid_n() {
        static int grid = 0;
        if (grid == 0) {
            cudaLaunchAttribute attr[1];
            cudaLaunchConfig_t cfg = xy_config<N, true>(attr, kXyCluster, nullptr);
            int nc0 = 0, nc1 = 0;
            if (set_smem(k_xy_cluster<N, kXyCluster, true>, cfg.dynamicSmemBytes) != cudaSuccess ||
                set_smem(k_xy_cluster<N, kXyCluster, false>, cfg.dynamicSmemBytes) != cudaSuccess ||
                cudaOccupancyMaxActiveClusters(&nc0, k_xy_cluster<N, kXyCluster, true>, &cfg) != cudaSuccess ||
                cudaOccupancyMaxActiveClusters(&nc1, k_xy_cluster<N, kXyCluster, false>, &cfg) != cudaSuccess)
                return 0;
            int nc = nc0 < nc1 ? nc0 : nc1;
            nc = nc < N ? nc : N;
            grid = nc * kXyCluster;
        }
        return grid;
    }
    template <int N, bool DO_YI>
    static cudaError_t xy_n(void* W, KgDev* dev, double* ps, double* pm, const void* tw, double scale, double lam,
                            cudaStream_t st) {
        const int grid = xy_grid_n<N>();
        if (grid < kXyCluster) return cudaErrorInvalidConfiguration;
        auto kern = k_xy_cluster<N, kXyCluster, DO_YI>;
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = xy_config<N, DO_YI>(attr, grid, st);
        cudaError_t e = set_smem(kern, cfg.dynamicSmemBytes);
        if (e != cudaSuccess) return e;
        return cudaLaunchKernelEx(&cfg, kern, (float2*)W, dev, ps, pm, (const float2*)tw, scale, lam);
    }
    static cudaError_t xy_fused(int N, int do_yi, void* W, KgDev* dev, double* ps, double* pm, const void* tw,
                                double scale, double lam, cudaStream_t st) {
        if constexpr (!std::is_same<P, PrecF32>::value) {
            return cudaErrorNotSupported;
        } else {
#define KG_XY_CASE(NN)                                                                       \
    case NN:                                                                                 \
        return do_yi ? xy_n<NN, true>(W, dev, ps, pm, tw, scale, lam, st)                    \
                     : xy_n<NN, false>(W, dev, ps, pm, tw, scale, lam, st);
            switch (N) {
                KG_XY_CASE(64)
                KG_XY_CASE(128)
                KG_XY_CASE(256)
                KG_XY_CASE(512)
                default: return cudaErrorNotSupported;
            }
#undef KG_XY_CASE
        }
    }
    static int xy_parts(int N) {
        if constexpr (!std::is_same<P, PrecF32>::value) {
            return 0;
        } else {
            switch (N) {
                case 64: return xy_grid_n<64>();
                case 128: return xy_grid_n<128>();
                case 256: return xy_grid_n<256>();
                case 512: return xy_grid_n<512>();
                default: return 0;
            }
        }
    }

    // the ensemble step (kg_ensemble.cuh); schedules differ in tile shape and stage order,
    // not in shared memory (a unit's tiles always hold 2048 values)
    template <int SCHED>
    static size_t ens_smem_s() {
        typedef EnsUnits<P, 64, SCHED> U64;
        typedef EnsUnits<P, 128, SCHED> U128;
        size_t a = (size_t)U64::LPU * XShape<64>::PADM, b = (size_t)U128::LPU * XShape<128>::PADM;
        size_t c = (size_t)U64::TPU * 64 * U64::C, d = (size_t)U128::TPU * 128 * U128::C;
        size_t m = a > b ? a : b;
        m = m > c ? m : c;
        m = m > d ? m : d;
        return m * sizeof(S);
    }
    template <int SCHED>
    static int ens_blocks_per_sm_s() {
        if (set_smem(k_ens_step<P, SCHED>, ens_smem_s<SCHED>()) != cudaSuccess) return 0;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ens_step<P, SCHED>, kEnsThreads, ens_smem_s<SCHED>()) !=
            cudaSuccess)
            return 0;
        return n;
    }
    static int ens_blocks_per_sm(int sched) {
        switch (sched) {
            case 0: return ens_blocks_per_sm_s<0>();
            case 1: return ens_blocks_per_sm_s<1>();
            case 2: return ens_blocks_per_sm_s<2>();
            case 3: return ens_blocks_per_sm_s<3>();
            default: return 0;
        }
    }
    template <int SCHED>
    static cudaError_t ens_step_s(const EnsParams& p, int grid, cudaStream_t st) {
        cudaError_t e = set_smem(k_ens_step<P, SCHED>, ens_smem_s<SCHED>());
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(kEnsThreads);
        cfg.dynamicSmemBytes = ens_smem_s<SCHED>();
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_ens_step<P, SCHED>, p);
    }
    static cudaError_t ens_step(const EnsParams& p, int grid, int sched, cudaStream_t st) {
        switch (sched) {
            case 0: return ens_step_s<0>(p, grid, st);
            case 1: return ens_step_s<1>(p, grid, st);
            case 2: return ens_step_s<2>(p, grid, st);
            case 3: return ens_step_s<3>(p, grid, st);
            default: return cudaErrorInvalidValue;
        }
    }
};

}  // namespace kg
