// kg_common.cu -- kernels every precision shares: the FP64 set-up and read-out
// transforms, the startup levels, the energy sums outside the recorded steps and the
// finalisers of a step.
#define KG_DEFINE_COMMON_KERNELS
#include "kg_launch_impl.cuh"

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

// Energy of the composed scheme at an integer step, quadratic part: per mode the velocity
// p = P + (h_0/2) G_{h_0}(uh) = P + (K_0 F - K_0 omega^2 uh) / 2 (kick0 holds (K_0, K_0 omega^2)),
// and the partial sums of w_k (|p|^2 + omega_k^2 |uh|^2) / 2 (Neumaier, per CTA)
template <int N>
__global__ void __launch_bounds__(256) k_energy_c4(const double2* __restrict__ a, const double2* __restrict__ P,
                                                   const double2* __restrict__ f, const double2* __restrict__ kick0,
                                                   const double* __restrict__ w2tab, double* __restrict__ part_sum) {
    typedef ModeIndex<N, false> MI;
    __shared__ double red[96];
    const size_t total = (size_t)MI::kModes;
    NSum acc;
    acc.s = 0.0;
    acc.c = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const MI mi((unsigned)i);
        const double w = mi.twice ? 2.0 : 1.0;
        const double2 kc = kick0[mi.m2], ai = a[i], pi = P[i], fi = f[i];
        const double pre = pi.x + 0.5 * (kc.x * fi.x - kc.y * ai.x);
        const double pim = pi.y + 0.5 * (kc.x * fi.y - kc.y * ai.y);
        acc.add(w * 0.5 * (pre * pre + pim * pim + w2tab[mi.m2] * (ai.x * ai.x + ai.y * ai.y)));
    }
    double mx = 0.0;
    block_reduce<256>(acc, mx, red);
    if (threadIdx.x == 0) part_sum[blockIdx.x] = acc.value();
}

cudaError_t launch_energy_c4(int N, const double2* a, const double2* P, const double2* f, const double2* kick0,
                             const double* w2tab, double* part_sum, int nparts, cudaStream_t st) {
    KG_DISPATCH_N(N, {
        k_energy_c4<NN><<<nparts, 256, 0, st>>>(a, P, f, kick0, w2tab, part_sum);
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
