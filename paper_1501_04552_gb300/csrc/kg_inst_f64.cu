// kg_inst_f64.cu -- pass launchers for the PrecF64 precision.
#define KG_DEFINE_COMMON_KERNELS
#include "kg_launch_impl.cuh"

namespace kg {
template struct Launchers<PrecF64>;
const PassLaunch kLaunchF64 = {
    &Launchers<PrecF64>::pass_x, &Launchers<PrecF64>::col, &Launchers<PrecF64>::col_from_f64, &Launchers<PrecF64>::update, &Launchers<PrecF64>::update_parts, &Launchers<PrecF64>::ens_step, &Launchers<PrecF64>::ens_blocks_per_sm, &Launchers<PrecF64>::x_parts, sizeof(PrecF64::S),
    &Launchers<PrecF64>::passc_x, &Launchers<PrecF64>::xc_parts, &Launchers<PrecF64>::colc, &Launchers<PrecF64>::colc_from_f64, &Launchers<PrecF64>::updatec, &Launchers<PrecF64>::updatec_parts,
    nullptr, nullptr,   // no fused z pass: the three-kernel form is faster for FP64
    nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
}  // namespace kg

namespace kg {

cudaError_t launch_x_forward(int N, const double* u, double2* out, const double2* tw, int cube, double lam,
                             cudaStream_t st) {
    KG_DISPATCH_N(N, {
        typedef XShape<NN> X;
        const size_t smem = (size_t)X::LPC * X::PADM * sizeof(double2);
        cudaError_t e = set_smem(k_x_forward<NN>, smem);
        if (e != cudaSuccess) return e;
        k_x_forward<NN><<<NN * NN / X::LPC, kXThreads, smem, st>>>(u, out, tw, cube, lam);
        return cudaGetLastError();
    });
}

cudaError_t launch_x_inverse(int N, const double2* in, double* u, const double2* tw, double scale, double* part_sum,
                             cudaStream_t st) {
    KG_DISPATCH_N(N, {
        typedef XShape<NN> X;
        const size_t smem = (size_t)X::LPC * X::PADM * sizeof(double2);
        cudaError_t e = set_smem(k_x_inverse<NN>, smem);
        if (e != cudaSuccess) return e;
        k_x_inverse<NN><<<NN * NN / X::LPC, kXThreads, smem, st>>>(in, u, tw, scale, part_sum);
        return cudaGetLastError();
    });
}

int x_inverse_parts(int N) { return N * N / (kXThreads / (N / 16)); }

cudaError_t launch_startup(int N, const double2* a, double2* b, const double2* f, const double2* coef, double dt,
                           bool cplx, cudaStream_t st) {
    KG_DISPATCH_N(N, {
        if (cplx) k_startup<NN, true><<<kStrideCtasDeep, 256, 0, st>>>(a, b, f, coef, dt);
        else k_startup<NN, false><<<kStrideCtasDeep, 256, 0, st>>>(a, b, f, coef, dt);
        return cudaGetLastError();
    });
}

cudaError_t launch_startup_c4(int N, const double2* a, double2* b, const double2* f, const double2* kick0,
                              cudaStream_t st) {
    KG_DISPATCH_N(N, {
        k_startup_c4<NN><<<kStrideCtasDeep, 256, 0, st>>>(a, b, f, kick0);
        return cudaGetLastError();
    });
}

cudaError_t launch_energy_q(int N, const double2* x, const double2* y, const double* w2tab, double inv_dt,
                            double* part_sum, int nparts, bool cplx, cudaStream_t st) {
    KG_DISPATCH_N(N, {
        if (cplx) k_energy_q<NN, true><<<nparts, 256, 0, st>>>(x, y, w2tab, inv_dt, part_sum);
        else k_energy_q<NN, false><<<nparts, 256, 0, st>>>(x, y, w2tab, inv_dt, part_sum);
        return cudaGetLastError();
    });
}

cudaError_t launch_xc_forward(int N, const double2* u, double2* out, const double2* tw, int cube, double lam,
                              cudaStream_t st) {
    KG_DISPATCH_N(N, {
        typedef XcShape<NN> X;
        const size_t smem = (size_t)X::LPC * X::PADN * sizeof(double2);
        cudaError_t e = set_smem(k_xc_forward<NN>, smem);
        if (e != cudaSuccess) return e;
        k_xc_forward<NN><<<NN * NN / X::LPC, kXThreads, smem, st>>>(u, out, tw, cube, lam);
        return cudaGetLastError();
    });
}

cudaError_t launch_xc_inverse(int N, const double2* in, double2* u, const double2* tw, double scale,
                              double* part_sum, cudaStream_t st) {
    KG_DISPATCH_N(N, {
        typedef XcShape<NN> X;
        const size_t smem = (size_t)X::LPC * X::PADN * sizeof(double2);
        cudaError_t e = set_smem(k_xc_inverse<NN>, smem);
        if (e != cudaSuccess) return e;
        k_xc_inverse<NN><<<NN * NN / X::LPC, kXThreads, smem, st>>>(in, u, tw, scale, part_sum);
        return cudaGetLastError();
    });
}

int xc_inverse_parts(int N) { return N * N / (kXThreads / (N / 8)); }

cudaError_t launch_fin_x(const double* ps, const double* pm, int count, KgDev* dev, double p_norm, cudaStream_t st) {
    k_fin_x<<<1, kFinThreads, 0, st>>>(ps, pm, count, dev, p_norm);
    return cudaGetLastError();
}

cudaError_t launch_fin_peek(const double* ps, const double* pm, int count, KgDev* dev, double p_norm,
                            cudaStream_t st) {
    k_fin_peek<<<1, kFinThreads, 0, st>>>(ps, pm, count, dev, p_norm);
    return cudaGetLastError();
}

cudaError_t launch_fin_z(const double* ps, int count, double* stage2, KgDev* dev, double q_norm, cudaStream_t st) {
    const int n2 = (count + kSumThreads - 1) / kSumThreads;
    k_sum_parts<<<n2, kSumThreads, 0, st>>>(ps, count, stage2, dev);
    k_fin_z<<<1, kFinThreads, 0, st>>>(stage2, n2, dev, q_norm);
    return cudaGetLastError();
}

cudaError_t launch_fin_sum(const double* ps, int count, double norm, double* out, cudaStream_t st) {
    k_fin_sum<<<1, kFinThreads, 0, st>>>(ps, count, norm, out);
    return cudaGetLastError();
}

}  // namespace kg
