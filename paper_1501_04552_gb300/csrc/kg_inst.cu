// kg_inst.cu -- one share of one precision's pass launchers (see kg_inst.h).
// Compiled with KG_PREC_ID = 0 (IEEE FP64), 1 (double-float) or 2 (FP32) and
// KG_PART = 0..4; each compile instantiates only the kernels of its share.
#include "kg_inst.h"
#include "kg_launch_impl.cuh"

#if !defined(KG_PREC_ID) || !defined(KG_PART)
#error "compile with -DKG_PREC_ID=<0|1|2> -DKG_PART=<0..4>"
#endif

#if KG_PREC_ID == 0
#define KG_P PrecF64
#define KG_NS inst_f64
#elif KG_PREC_ID == 1
#define KG_P PrecDF
#define KG_NS inst_df
#else
#define KG_P PrecF32
#define KG_NS inst_f32
#endif

namespace kg {
namespace KG_NS {
typedef Launchers<KG_P> Lp;

#if KG_PART == 0
cudaError_t pass_x(int N, int mode, void* W, KgDev* dev, double* ps, double* pm, const void* tw, double scale,
                   double lam, cudaStream_t st) {
    return Lp::pass_x(N, mode, W, dev, ps, pm, tw, scale, lam, st);
}
int x_parts(int N) { return Lp::x_parts(N); }
cudaError_t x_setup(int N, const double* u, void* spec, const void* tw, int cube, double lam, cudaStream_t st) {
    return Lp::x_setup(N, u, spec, tw, cube, lam, st);
}
cudaError_t x_readout(int N, void* spec, double* u, const void* tw, double scale, cudaStream_t st) {
    return Lp::x_readout(N, spec, u, tw, scale, st);
}
cudaError_t xy_fused(int N, int do_yi, void* W, KgDev* dev, double* ps, double* pm, const void* tw, double scale,
                     double lam, cudaStream_t st) {
    return Lp::xy_fused(N, do_yi, W, dev, ps, pm, tw, scale, lam, st);
}
int xy_parts(int N) { return Lp::xy_parts(N); }
#elif KG_PART == 1
cudaError_t col(int N, int sign, void* W, size_t ps, size_t rs, int nplanes, const void* tw, cudaStream_t st) {
    return Lp::col(N, sign, W, ps, rs, nplanes, tw, st);
}
cudaError_t col_from_f64(int N, const double2* src0, const double2* src1, const KgDev* dev, void* W, size_t ps,
                         size_t rs, int nplanes, const void* tw, cudaStream_t st) {
    return Lp::col_from_f64(N, src0, src1, dev, W, ps, rs, nplanes, tw, st);
}
cudaError_t col_to_f64(int N, const void* W, double2* out, size_t ps, size_t rs, int nplanes, const void* tw,
                       cudaStream_t st) {
    return Lp::col_to_f64(N, W, out, ps, rs, nplanes, tw, st);
}
#elif KG_PART == 2
cudaError_t zstep(int N, bool cplx, void* W, double2* S0, double2* S1, KgDev* dev, double* ps, const void* tw,
                  const double2* coef, const double* w2, double inv_dt, const C4Args* c4, cudaStream_t st) {
#if KG_PREC_ID == 0
    // the IEEE FP64 step runs forward z, update and inverse z as three kernels
    (void)N, (void)cplx, (void)W, (void)S0, (void)S1, (void)dev, (void)ps, (void)tw, (void)coef, (void)w2;
    (void)inv_dt, (void)c4, (void)st;
    return cudaErrorNotSupported;
#else
    return Lp::zstep(N, cplx, W, S0, S1, dev, ps, tw, coef, w2, inv_dt, c4, st);
#endif
}
int zstep_parts(int N, bool cplx) { return Lp::zstep_parts(N, cplx); }
cudaError_t update(int N, void* W, double2* S0, double2* S1, KgDev* dev, double* ps, const double2* coef,
                   const double* w2, double inv_dt, const C4Args* c4, cudaStream_t st) {
    return Lp::update(N, W, S0, S1, dev, ps, coef, w2, inv_dt, c4, st);
}
int update_parts(int N) { return Lp::update_parts(N); }
#elif KG_PART == 3
cudaError_t passc_x(int N, int mode, void* W, KgDev* dev, double* ps, double* pm, const void* tw, double scale,
                    double lam, cudaStream_t st) {
    return Lp::passc_x(N, mode, W, dev, ps, pm, tw, scale, lam, st);
}
int xc_parts(int N) { return Lp::xc_parts(N); }
cudaError_t colc(int N, int sign, void* W, size_t ps, size_t rs, int nplanes, const void* tw, cudaStream_t st) {
    return Lp::colc(N, sign, W, ps, rs, nplanes, tw, st);
}
cudaError_t colc_from_f64(int N, const double2* src0, const double2* src1, const KgDev* dev, void* W, size_t ps,
                          size_t rs, int nplanes, const void* tw, cudaStream_t st) {
    return Lp::colc_from_f64(N, src0, src1, dev, W, ps, rs, nplanes, tw, st);
}
cudaError_t updatec(int N, void* W, double2* S0, double2* S1, KgDev* dev, double* ps, const double2* coef,
                    const double* w2, double inv_dt, cudaStream_t st) {
    return Lp::updatec(N, W, S0, S1, dev, ps, coef, w2, inv_dt, st);
}
int updatec_parts(int N) { return Lp::updatec_parts(N); }
cudaError_t xc_setup(int N, const double2* u, void* spec, const void* tw, int cube, double lam, cudaStream_t st) {
    return Lp::xc_setup(N, u, spec, tw, cube, lam, st);
}
cudaError_t xc_readout(int N, void* spec, double2* u, const void* tw, double scale, cudaStream_t st) {
    return Lp::xc_readout(N, spec, u, tw, scale, st);
}
cudaError_t colc_to_f64(int N, const void* W, double2* out, size_t ps, size_t rs, int nplanes, const void* tw,
                        cudaStream_t st) {
    return Lp::colc_to_f64(N, W, out, ps, rs, nplanes, tw, st);
}
#elif KG_PART == 4
cudaError_t ens_step(const EnsParams& p, int grid, int sched, cudaStream_t st) {
    return Lp::ens_step(p, grid, sched, st);
}
int ens_blocks_per_sm(int sched) { return Lp::ens_blocks_per_sm(sched); }
#else
#error "KG_PART out of range"
#endif

}  // namespace KG_NS
}  // namespace kg
