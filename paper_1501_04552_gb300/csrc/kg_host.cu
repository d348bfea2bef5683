// kg_host.cu -- host helpers shared by the single-state context and the ensemble:
// the per-grid tables and the FP64 set-up of a state (startup level of the scheme).
#include <cmath>
#include <vector>

#include "../../include/kg.h"
#include "kg_launch.h"

namespace kg {

namespace {
const double kPi = 3.14159265358979323846;

#define KG_HCK(call)                                                                                 \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return set_last_error(KG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// FP64 R2C of a physical device array into out; cube: lam u^3 instead of u
int forward3d(int N, const double* u, double2* out, const double2* tw64, int cube, double lam, cudaStream_t st) {
    const int NH = N / 2 + 1;
    KG_HCK(launch_x_forward(N, u, out, tw64, cube, lam, st));
    KG_HCK(kLaunchF64.col(N, -1, out, (size_t)N * NH, NH, N, tw64, st));   // y
    KG_HCK(kLaunchF64.col(N, -1, out, NH, (size_t)N * NH, N, tw64, st));   // z
    return KG_OK;
}
// FP64 forward 3D transform of a complex physical device array (full spectrum);
// cube: of lam |u|^2 u instead of u
int forward3d_c(int N, const double2* u, double2* out, const double2* tw64, int cube, double lam, cudaStream_t st) {
    KG_HCK(launch_xc_forward(N, u, out, tw64, cube, lam, st));
    KG_HCK(kLaunchF64.colc(N, -1, out, (size_t)N * N, N, N, tw64, st));   // y
    KG_HCK(kLaunchF64.colc(N, -1, out, N, (size_t)N * N, N, tw64, st));   // z
    return KG_OK;
}
// forward 3D transform of a physical FP64 array in the pass precision of pl, W as the
// work array, into the FP64 spectral array out; cube: of lam u^3 instead of u
int forward3d_pass(int N, const PassLaunch* pl, const double* u, void* W, double2* out, const void* tw, int cube,
                   double lam, cudaStream_t st) {
    const int NH = N / 2 + 1;
    KG_HCK(pl->x_setup(N, u, W, tw, cube, lam, st));
    KG_HCK(pl->col(N, -1, W, (size_t)N * NH, NH, N, tw, st));             // y
    KG_HCK(pl->col_to_f64(N, W, out, NH, (size_t)N * NH, N, tw, st));     // z -> FP64
    return KG_OK;
}
// the same for a complex physical field (full spectrum)
int forward3d_c_pass(int N, const PassLaunch* pl, const double2* u, void* W, double2* out, const void* tw, int cube,
                     double lam, cudaStream_t st) {
    KG_HCK(pl->xc_setup(N, u, W, tw, cube, lam, st));
    KG_HCK(pl->colc(N, -1, W, (size_t)N * N, N, N, tw, st));              // y
    KG_HCK(pl->colc_to_f64(N, W, out, N, (size_t)N * N, N, tw, st));      // z -> FP64
    return KG_OK;
}
}  // namespace

int forward3d_f64(int N, const double* u, double2* out, const double2* tw64, int cube, double lam, cudaStream_t st) {
    return forward3d(N, u, out, tw64, cube, lam, st);
}

const PassLaunch* launcher_for(int prec) {
    switch (prec) {
        case KG_FP64: return &kLaunchF64;
        case KG_DF64: return &kLaunchDF;
        case KG_MIXED: return &kLaunchF32;
        default: return nullptr;
    }
}

int make_tables(int N, int prec, double L, double dt, const AllocFn& alloc, Tables* t) {
    std::vector<double2> t64(N);
    for (int j = 0; j < N; j++) {
        const double a = 2.0 * kPi * (double)j / (double)N;
        t64[j] = make_double2(std::cos(a), -std::sin(a));
    }
    int rc = alloc((void**)&t->tw64, sizeof(double2) * N, "twiddles fp64");
    if (rc) return rc;
    KG_HCK(cudaMemcpy(t->tw64, t64.data(), sizeof(double2) * N, cudaMemcpyHostToDevice));
    if (prec == KG_FP64) {
        t->tw = t->tw64;
    } else if (prec == KG_DF64) {
        std::vector<float4> v(N);
        for (int j = 0; j < N; j++) {
            const float rh = (float)t64[j].x, ih = (float)t64[j].y;
            // (re.hi, im.hi, re.lo, im.lo), the layout of a double-float value (PrecDF::S)
            v[j] = make_float4(rh, ih, (float)(t64[j].x - (double)rh), (float)(t64[j].y - (double)ih));
        }
        rc = alloc(&t->tw, sizeof(float4) * N, "twiddles df");
        if (rc) return rc;
        KG_HCK(cudaMemcpy(t->tw, v.data(), sizeof(float4) * N, cudaMemcpyHostToDevice));
    } else {
        std::vector<float2> v(N);
        for (int j = 0; j < N; j++) v[j] = make_float2((float)t64[j].x, (float)t64[j].y);
        rc = alloc(&t->tw, sizeof(float2) * N, "twiddles f32");
        if (rc) return rc;
        KG_HCK(cudaMemcpy(t->tw, v.data(), sizeof(float2) * N, cudaMemcpyHostToDevice));
    }
    // coefficients of Eq. (2) by integer wavenumber norm m^2 = mx^2 + my^2 + mz^2
    const int m2max = 3 * (N / 2) * (N / 2);
    std::vector<double2> cf(m2max + 1);
    std::vector<double> w2(m2max + 1);
    const double kf = 2.0 * kPi / L;
    for (int m2 = 0; m2 <= m2max; m2++) {
        const double om2 = 1.0 + kf * kf * (double)m2;
        const double a = dt * dt * om2 / 4.0;
        const double cc = (1.0 - a) / (1.0 + a);
        const double beta = (dt * dt / 2.0) / (1.0 + a);
        cf[m2] = make_double2(2.0 * cc, 2.0 * beta);
        w2[m2] = om2;
    }
    rc = alloc((void**)&t->coef, sizeof(double2) * (m2max + 1), "coefficients");
    if (rc) return rc;
    rc = alloc((void**)&t->w2, sizeof(double) * (m2max + 1), "omega^2");
    if (rc) return rc;
    KG_HCK(cudaMemcpy(t->coef, cf.data(), sizeof(double2) * (m2max + 1), cudaMemcpyHostToDevice));
    KG_HCK(cudaMemcpy(t->w2, w2.data(), sizeof(double) * (m2max + 1), cudaMemcpyHostToDevice));
    return KG_OK;
}

// composed scheme (triple jump of Eq. (2) in kick-drift-kick form): substep lengths
// h = (g1, g2, g1) dt, g1 = 1/(2 - 2^{1/3}), g2 = 1 - 2 g1, and per substep s the merged
// kick K_s = half(h_{s-1}) + half(h_s), half(h) = (h/2)/(1 + omega^2 h^2/4), h_{-1} = h_2
int make_kick_tables(int N, double L, double dt, const AllocFn& alloc, double2** kick, double h[3]) {
    const double g1 = 1.0 / (2.0 - std::cbrt(2.0)), g2 = 1.0 - 2.0 * g1;
    h[0] = g1 * dt;
    h[1] = g2 * dt;
    h[2] = g1 * dt;
    const int m2max = 3 * (N / 2) * (N / 2), stride = m2max + 1;
    std::vector<double2> t((size_t)3 * stride);
    const double kf = 2.0 * kPi / L;
    for (int m2 = 0; m2 <= m2max; m2++) {
        const double om2 = 1.0 + kf * kf * (double)m2;
        auto half = [om2](double hs) { return (0.5 * hs) / (1.0 + om2 * hs * hs / 4.0); };
        for (int s = 0; s < 3; s++) {
            const double K = half(h[(s + 2) % 3]) + half(h[s]);
            t[(size_t)s * stride + m2] = make_double2(K, K * om2);
        }
    }
    int rc = alloc((void**)kick, sizeof(double2) * t.size(), "composed-scheme kick tables");
    if (rc) return rc;
    KG_HCK(cudaMemcpy(*kick, t.data(), sizeof(double2) * t.size(), cudaMemcpyHostToDevice));
    return KG_OK;
}

int init_state(int N, int prec, double dt, double lam, const Tables& tb, double* phys, const double* v0,
               bool v0_on_device, double2* S0, double2* S1, void* W, double2* fbuf, cudaStream_t st,
               const double2* kick0, bool pass_precision) {
    const int NH = N / 2 + 1;
    const size_t nspec = (size_t)N * N * NH, n3 = (size_t)N * N * N;
    const PassLaunch* pl = launcher_for(prec);
    if (!pl) return set_last_error(KG_EINVAL, "unknown precision");
    const bool pass = pass_precision && pl->x_setup != nullptr;
    auto fwd = [&](double2* out, int cube) {
        return pass ? forward3d_pass(N, pl, phys, W, out, tb.tw, cube, lam, st)
                    : forward3d(N, phys, out, tb.tw64, cube, lam, st);
    };
    int rc = fwd(fbuf, 1);              // F^0 = R2C(lam u0^3)
    if (!rc) rc = fwd(S0, 0);           // uh^0
    if (rc) return rc;
    if (v0) {
        KG_HCK(cudaMemcpyAsync(phys, v0, sizeof(double) * n3, v0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        rc = fwd(S1, 0);                // vh^0
        if (rc) return rc;
    } else {
        KG_HCK(cudaMemsetAsync(S1, 0, sizeof(double2) * nspec, st));
    }
    if (kick0) KG_HCK(launch_startup_c4(N, S0, S1, fbuf, kick0, st));    // S1 = P^0
    else KG_HCK(launch_startup(N, S0, S1, fbuf, tb.coef, dt, false, st));  // S1 = uh^{-1}
    KG_HCK(pl->col_from_f64(N, S0, S1, nullptr, W, NH, (size_t)N * NH, N, tb.tw, st));   // z inverse of uh^0
    KG_HCK(pl->col(N, +1, W, (size_t)N * NH, NH, N, tb.tw, st));                          // y inverse
    return KG_OK;
}

int init_state_c(int N, int prec, double dt, double lam, const Tables& tb, double2* phys, const double2* v0,
                 bool v0_on_device, double2* S0, double2* S1, void* W, double2* fbuf, cudaStream_t st,
                 bool pass_precision) {
    const size_t n3 = (size_t)N * N * N;
    const PassLaunch* pl = launcher_for(prec);
    if (!pl) return set_last_error(KG_EINVAL, "unknown precision");
    const bool pass = pass_precision && pl->xc_setup != nullptr;
    auto fwd = [&](double2* out, int cube) {
        return pass ? forward3d_c_pass(N, pl, phys, W, out, tb.tw, cube, lam, st)
                    : forward3d_c(N, phys, out, tb.tw64, cube, lam, st);
    };
    int rc = fwd(fbuf, 1);              // F^0 = FFT(lam |u0|^2 u0)
    if (!rc) rc = fwd(S0, 0);           // uh^0
    if (rc) return rc;
    if (v0) {
        KG_HCK(cudaMemcpyAsync(phys, v0, sizeof(double2) * n3, v0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        rc = fwd(S1, 0);                // vh^0
        if (rc) return rc;
    } else {
        KG_HCK(cudaMemsetAsync(S1, 0, sizeof(double2) * n3, st));
    }
    KG_HCK(launch_startup(N, S0, S1, fbuf, tb.coef, dt, true, st));       // S1 = uh^{-1}
    KG_HCK(pl->colc_from_f64(N, S0, S1, nullptr, W, N, (size_t)N * N, N, tb.tw, st));   // z inverse of uh^0
    KG_HCK(pl->colc(N, +1, W, (size_t)N * N, N, N, tb.tw, st));                         // y inverse
    return KG_OK;
}

}  // namespace kg
