// kg_launch.h -- host-side launchers of the step passes (one definition per precision).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <functional>
#include <string>

namespace kg {

// grid sizes of the grid-stride kernels (any count is correct; these fill a 152-SM GB300
// four or eight CTAs deep)
constexpr int kStrideCtas = 152 * 4;
constexpr int kStrideCtasDeep = 152 * 8;

struct KgDev;
struct EnsParams;

// the composed scheme's per-substep data, passed by value to the update kernels
struct C4Args {
    const double2* kick;   // [3][stride]: (K_s, K_s omega^2) by integer m^2
    int stride;            // entries per substep table (3 (N/2)^2 + 1)
    double h[3];           // drift length of each substep
};

// precision ids match KG_FP64 / KG_DF64 / KG_MIXED of kg.h
struct PassLaunch {
    // x pass over W in the context's precision; mode 0 step, 1 peek.  Writes nparts partials.
    cudaError_t (*pass_x)(int N, int mode, void* W, KgDev* dev, double* part_sum, double* part_max, const void* tw,
                          double scale, double lam, cudaStream_t st);
    // column FFT in place on W (sign -1 forward, +1 inverse)
    cudaError_t (*col)(int N, int sign, void* W, size_t plane_stride, size_t row_stride, int nplanes, const void* tw,
                       cudaStream_t st);
    // inverse column FFT from an FP64 spectral source (chosen by dev->phase when src1 != NULL) into W
    cudaError_t (*col_from_f64)(int N, const double2* src0, const double2* src1, const KgDev* dev, void* W,
                                size_t plane_stride, size_t row_stride, int nplanes, const void* tw, cudaStream_t st);
    // streaming FP64 update between a forward and an inverse z column pass; writes
    // update_parts(N) Q partials when recording; c4: the composed scheme's tables (NULL:
    // Eq. (2))
    cudaError_t (*update)(int N, void* W, double2* S0, double2* S1, KgDev* dev, double* part_sum, const double2* coef,
                          const double* w2tab, double inv_dt, const C4Args* c4, cudaStream_t st);
    int (*update_parts)(int N);
    // one persistent cooperative launch of an ensemble step (kg_ensemble.cuh) in launch
    // schedule sched (0 .. kEnsSchedules-1), and the CTAs per SM that schedule can hold
    cudaError_t (*ens_step)(const EnsParams& p, int grid, int sched, cudaStream_t st);
    int (*ens_blocks_per_sm)(int sched);
    int (*x_parts)(int N);
    size_t store_bytes;  // bytes of one complex value of W
    // complex field (full N^3 spectrum, N columns per plane): x pass, column FFTs,
    // column FFT from an FP64 source, update, and their partial counts
    cudaError_t (*passc_x)(int N, int mode, void* W, KgDev* dev, double* part_sum, double* part_max, const void* tw,
                           double scale, double lam, cudaStream_t st);
    int (*xc_parts)(int N);
    cudaError_t (*colc)(int N, int sign, void* W, size_t plane_stride, size_t row_stride, int nplanes, const void* tw,
                        cudaStream_t st);
    cudaError_t (*colc_from_f64)(int N, const double2* src0, const double2* src1, const KgDev* dev, void* W,
                                 size_t plane_stride, size_t row_stride, int nplanes, const void* tw, cudaStream_t st);
    cudaError_t (*updatec)(int N, void* W, double2* S0, double2* S1, KgDev* dev, double* part_sum,
                           const double2* coef, const double* w2tab, double inv_dt, cudaStream_t st);
    int (*updatec_parts)(int N);
    // the z pass in one kernel: forward z FFT, update (as update / updatec), inverse z
    // FFT, of a real (cplx = false) or complex field; zstep_parts(N, cplx) Q partials.
    // NULL where the step runs forward z, update and inverse z as three kernels.
    cudaError_t (*zstep)(int N, bool cplx, void* W, double2* S0, double2* S1, KgDev* dev, double* part_sum,
                         const void* tw, const double2* coef, const double* w2tab, double inv_dt, const C4Args* c4,
                         cudaStream_t st);
    int (*zstep_parts)(int N, bool cplx);
    // set-up and read-out transforms in the pass precision (NULL: the FP64 kernels serve):
    // x_setup: physical FP64 lines (lam u^3 when cube) -> half spectra along x in W format;
    // x_readout: W-format half spectra along x -> physical FP64 lines times scale;
    // col_to_f64: forward column FFT of a W-format array into an FP64 spectral array
    cudaError_t (*x_setup)(int N, const double* u, void* spec, const void* tw, int cube, double lam, cudaStream_t st);
    cudaError_t (*x_readout)(int N, void* spec, double* u, const void* tw, double scale, cudaStream_t st);
    cudaError_t (*col_to_f64)(int N, const void* W, double2* out, size_t plane_stride, size_t row_stride,
                              int nplanes, const void* tw, cudaStream_t st);
    // the same for a complex field (N-point lines, N columns per plane)
    cudaError_t (*xc_setup)(int N, const double2* u, void* spec, const void* tw, int cube, double lam,
                            cudaStream_t st);
    cudaError_t (*xc_readout)(int N, void* spec, double2* u, const void* tw, double scale, cudaStream_t st);
    cudaError_t (*colc_to_f64)(int N, const void* W, double2* out, size_t plane_stride, size_t row_stride,
                               int nplanes, const void* tw, cudaStream_t st);
    // inverse y, x pass and forward y of every z-plane in one launch of thread-block
    // clusters (kg_xyfuse.cuh; NULL where not built): do_yi = 0 leaves out the inverse y
    // transforms (W already holds the y-inverse); writes xy_parts(N) partials of the x
    // pass's statistics; cudaErrorNotSupported for grids it is not built for
    cudaError_t (*xy_fused)(int N, int do_yi, void* W, KgDev* dev, double* part_sum, double* part_max,
                            const void* tw, double scale, double lam, cudaStream_t st);
    int (*xy_parts)(int N);
};

extern const PassLaunch kLaunchF64;
extern const PassLaunch kLaunchDF;
extern const PassLaunch kLaunchF32;

// FP64 set-up / read-out launchers
cudaError_t launch_x_forward(int N, const double* u, double2* out, const double2* tw, int cube, double lam,
                             cudaStream_t st);
cudaError_t launch_x_inverse(int N, const double2* in, double* u, const double2* tw, double scale, double* part_sum,
                             cudaStream_t st);
int x_inverse_parts(int N);   // partial sums launch_x_inverse writes
// cplx: full N^3 spectrum of a complex field instead of the half spectrum
cudaError_t launch_startup(int N, const double2* a, double2* b, const double2* f, const double2* coef, double dt,
                           bool cplx, cudaStream_t st);
// startup of the composed scheme (real field): b = vh^0 -> P^0 (k_startup_c4)
cudaError_t launch_startup_c4(int N, const double2* a, double2* b, const double2* f, const double2* kick0,
                              cudaStream_t st);
cudaError_t launch_energy_q(int N, const double2* x, const double2* y, const double* w2tab, double inv_dt,
                            double* part_sum, int nparts, bool cplx, cudaStream_t st);
// complex field, FP64: forward transform along x (u -> out; cube: of lam |u|^2 u) and
// inverse transform along x times scale (u may be NULL; part_sum: per-CTA sum |u|^4)
cudaError_t launch_xc_forward(int N, const double2* u, double2* out, const double2* tw, int cube, double lam,
                              cudaStream_t st);
cudaError_t launch_xc_inverse(int N, const double2* in, double2* u, const double2* tw, double scale,
                              double* part_sum, cudaStream_t st);
int xc_inverse_parts(int N);
cudaError_t launch_fin_x(const double* ps, const double* pm, int count, KgDev* dev, double p_norm, cudaStream_t st);
cudaError_t launch_fin_peek(const double* ps, const double* pm, int count, KgDev* dev, double p_norm,
                            cudaStream_t st);
// after the update: Q from its count partials (summed pairwise in blocks of 1024 into
// stage2, which holds (count + 1023) / 1024 doubles), then the level/phase advance
cudaError_t launch_fin_z(const double* ps, int count, double* stage2, KgDev* dev, double q_norm, cudaStream_t st);
cudaError_t launch_fin_sum(const double* ps, int count, double norm, double* out, cudaStream_t st);
// composed scheme: partials of the quadratic energy sum_k w_k (|p|^2 + omega^2 |a|^2) / 2 with
// the synchronised velocity p formed from the stored P, F = R2C(lam u^3) and the first kick table
cudaError_t launch_energy_c4(int N, const double2* a, const double2* P, const double2* f, const double2* kick0,
                             const double* w2tab, double* part_sum, int nparts, cudaStream_t st);
// FP64 forward 3D transform of a physical array (cube: of lam u^3 instead of u)
int forward3d_f64(int N, const double* u, double2* out, const double2* tw64, int cube, double lam, cudaStream_t st);

// ---------------------------------------------------------------------------
// shared host helpers (kg_host.cu)
// ---------------------------------------------------------------------------
const PassLaunch* launcher_for(int prec);

// device tables of one grid: twiddles exp(-2 pi i j/N) in the pass precision and in
// FP64, (2 c_k, 2 beta_k) and omega_k^2 by integer m^2 = mx^2 + my^2 + mz^2
struct Tables {
    void* tw;
    double2* tw64;
    double2* coef;
    double* w2;
};
typedef std::function<int(void**, size_t, const char*)> AllocFn;
int make_tables(int N, int prec, double L, double dt, const AllocFn& alloc, Tables* t);
// the composed scheme's merged-kick tables [3][3 (N/2)^2 + 1] of (K_s, K_s omega^2) and
// its substep lengths h[3] = (g1, g2, g1) dt
int make_kick_tables(int N, double L, double dt, const AllocFn& alloc, double2** kick, double h[3]);

// Set-up of one state from the physical field in phys (N^3 doubles, overwritten):
// S0 = uh^0, S1 = uh^{-1} (startup level of Eq. (2)) or, with kick0 (the composed
// scheme's first merged-kick table), S1 = P^0; W = yz-inverse of uh^0 in the pass
// precision; fbuf is an FP64 spectral scratch (may alias W when W holds 16-byte values,
// unless pass_precision).  The transforms run in FP64, or with pass_precision (and a
// precision that has x_setup) in the pass precision with W as their work array.
int init_state(int N, int prec, double dt, double lam, const Tables& tb, double* phys, const double* v0,
               bool v0_on_device, double2* S0, double2* S1, void* W, double2* fbuf, cudaStream_t st,
               const double2* kick0 = nullptr, bool pass_precision = false);

// the same for a complex field: phys and v0 hold N^3 complex values, S0, S1, W and fbuf
// the full N^3 spectrum
int init_state_c(int N, int prec, double dt, double lam, const Tables& tb, double2* phys, const double2* v0,
                 bool v0_on_device, double2* S0, double2* S1, void* W, double2* fbuf, cudaStream_t st,
                 bool pass_precision = false);

// record a failure for kg_last_error(); returns code
int set_last_error(int code, const std::string& msg);

}  // namespace kg
