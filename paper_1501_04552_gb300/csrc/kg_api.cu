// kg_api.cu -- the C ABI of include/kg.h: context, set-up, stepping, energy, read-out.
//
// The scheme is Eq. (2) of Aseeri et al. (section 1.1.2) stepped in Fourier space;
// the energy is the discrete counterpart of the functional of section 1.1 stated in
// kg.h.  Host code only sequences passes, keeps tables and moves data; every step of
// the method runs in the kernels of kg_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/kg.h"

static_assert(sizeof(kg_state_header) == 256, "checkpoint header layout");
#include "kg_fft.cuh"
#include "kg_launch.h"

using namespace kg;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define KG_CK(call)                                                                              \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return fail(KG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)


bool supported_n(int N) { return N == 16 || N == 32 || N == 64 || N == 128 || N == 256 || N == 512; }

const PassLaunch* launcher(int prec) { return launcher_for(prec); }

// Test hook: KG_TEST_FAIL_ALLOC=k makes the k-th device allocation of a set-up fail
// (counted from 1), so the error path and its clean-up can be exercised on the host.
int g_alloc_counter = 0;

struct Ctx {
    int N = 0, NH = 0, prec = KG_DF64;
    bool cplx = false;       // complex field: full N^3 spectrum, N columns per plane
    double L = 0, dt = 0, lam = 1.0;
    size_t nspec = 0, nphys = 0;   // complex values per spectral array, reals per physical array
    cudaStream_t own_stream = nullptr;
    const PassLaunch* pl = nullptr;
    double2* S0 = nullptr;   // FP64 state arrays; dev->phase tells which holds uh^n
    double2* S1 = nullptr;
    void* W = nullptr;       // work array in the pass precision
    double2* tmp = nullptr;  // FP64 spectral scratch (set-up and read-out), allocated on demand
    double* phys = nullptr;  // physical scratch (N^3 doubles), on demand
    KgDev* dev = nullptr;
    double* part_sum = nullptr;
    double* part_max = nullptr;
    double* part2 = nullptr;  // second-stage partial sums of the update's Q
    int nparts = 0;
    double* scal = nullptr;  // device scalars for on-demand sums
    void* tw = nullptr;      // twiddles exp(-2 pi i j/N), j < N, in the pass precision
    double2* tw64 = nullptr; // same in FP64 for set-up and read-out
    double2* coef = nullptr; // (2 c, 2 beta) by integer m^2
    double* w2 = nullptr;    // omega^2 by integer m^2
    int scheme = KG_SCHEME_EQ2;
    double2* kick = nullptr; // composed scheme: merged-kick tables [3][m2max + 1]
    double c4h[3] = {0.0, 0.0, 0.0};   // composed scheme: substep lengths
    std::vector<void*> allocs;
    size_t bytes = 0;
    bool have_E0 = false;
    double E0 = 0.0;
    cudaEvent_t ev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaGraphExec_t step_graph = nullptr;   // one captured step, replayed by kg_step
    cudaGraphExec_t xy_graph = nullptr;     // one captured step of the fused xy form (inverse y included)
    long long launched = 0;                 // steps enqueued so far
    bool plain_done = false;                // a step of the separate-pass form ran outside a graph
    bool x_ahead = false;                   // kg_energy ran the next step's x pass (kg_step skips it)
    long long e_level = -1;                 // level of the last kg_energy result, and the result
    double e_value = 0.0;
};

Ctx* g_ctx = nullptr;
kg_options g_opt = {KG_DF64, 0, 1.0, 0.0, 0.0, nullptr};
int g_scheme = KG_SCHEME_EQ2;
int g_xy_fusion = 0;   // kg_set_xy_fusion
cudaStream_t g_user_stream = nullptr;

cudaStream_t stream_of(const Ctx* c) { return g_user_stream ? g_user_stream : c->own_stream; }

int dalloc(Ctx* c, void** p, size_t bytes, const char* what) {
    const char* inj = std::getenv("KG_TEST_FAIL_ALLOC");
    ++g_alloc_counter;
    if (inj && std::atoi(inj) == g_alloc_counter) {
        *p = nullptr;
        return fail(KG_ENOMEM, std::string("injected allocation failure: ") + what);
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(KG_ENOMEM, std::string("cudaMalloc(") + what + ", " + std::to_string(bytes) + " B): " +
                                   cudaGetErrorString(e));
    }
    c->allocs.push_back(*p);
    c->bytes += bytes;
    return KG_OK;
}

void destroy(Ctx* c) {
    if (!c) return;
    if (c->own_stream) cudaStreamSynchronize(c->own_stream);
    if (g_user_stream) cudaStreamSynchronize(g_user_stream);
    for (void* p : c->allocs) cudaFree(p);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->step_graph) cudaGraphExecDestroy(c->step_graph);
    if (c->xy_graph) cudaGraphExecDestroy(c->xy_graph);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

int upload_tables(Ctx* c) {
    Tables t;
    int rc = make_tables(c->N, c->prec, c->L, c->dt,
                         [c](void** p, size_t b, const char* w) { return dalloc(c, p, b, w); }, &t);
    if (rc) return rc;
    c->tw = t.tw;
    c->tw64 = t.tw64;
    c->coef = t.coef;
    c->w2 = t.w2;
    if (!c->cplx) {
        rc = make_kick_tables(c->N, c->L, c->dt, [c](void** p, size_t b, const char* w) { return dalloc(c, p, b, w); },
                              &c->kick, c->c4h);
        if (rc) return rc;
    }
    return KG_OK;
}

int ensure_scratch(Ctx* c) {
    int rc = KG_OK;
    if (!c->tmp) rc = dalloc(c, (void**)&c->tmp, sizeof(double2) * c->nspec, "fp64 spectral scratch");
    if (!rc && !c->phys) rc = dalloc(c, (void**)&c->phys, sizeof(double) * c->nphys, "physical scratch");
    return rc;
}

// FP64 inverse of a spectral state array (phase-selected pair) into c->tmp (yz only)
int inverse_yz_f64(Ctx* c, const double2* src0, const double2* src1, const KgDev* sel) {
    const int N = c->N, NH = c->NH;
    cudaStream_t st = stream_of(c);
    if (c->cplx) {
        KG_CK(kLaunchF64.colc_from_f64(N, src0, src1, sel, c->tmp, N, (size_t)N * N, N, c->tw64, st));   // z
        KG_CK(kLaunchF64.colc(N, +1, c->tmp, (size_t)N * N, N, N, c->tw64, st));                        // y
        return KG_OK;
    }
    KG_CK(kLaunchF64.col_from_f64(N, src0, src1, sel, c->tmp, NH, (size_t)N * NH, N, c->tw64, st));   // z
    KG_CK(kLaunchF64.col(N, +1, c->tmp, (size_t)N * NH, NH, N, c->tw64, st));                         // y
    return KG_OK;
}

double inv_n3(int N) { return 1.0 / ((double)N * (double)N * (double)N); }

// 1 if a[0..n) holds an infinity or a NaN: exponent field all ones, tested on the bit
// patterns without branches so the loop vectorises
int nonfinite_in(const double* a, size_t n) {
    unsigned long long bad = 0;
    for (size_t i = 0; i < n; i++) {
        unsigned long long b;
        std::memcpy(&b, a + i, 8);
        bad |= (unsigned long long)((b & 0x7FF0000000000000ull) == 0x7FF0000000000000ull);
    }
    return bad != 0;
}

// host-side check of an input field; large fields are split across host threads
int check_finite(const double* a, size_t n, const char* what) {
    const size_t kChunk = (size_t)1 << 22;
    int bad = 0;
    if (n <= kChunk) {
        bad = nonfinite_in(a, n);
    } else {
        const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        const size_t per = (n + hw - 1) / hw;
        std::vector<int> flags(hw, 0);
        std::vector<std::thread> pool;
        for (unsigned t = 0; t < hw; t++) {
            const size_t lo = std::min(n, (size_t)t * per), hi = std::min(n, lo + per);
            pool.emplace_back([a, lo, hi, t, &flags] { flags[t] = nonfinite_in(a + lo, hi - lo); });
        }
        for (auto& th : pool) th.join();
        for (int f : flags) bad |= f;
    }
    if (bad) return fail(KG_EINVAL, std::string(what) + " has a non-finite entry");
    return KG_OK;
}

int check_grid(int N, double L, double dt) {
    if (!supported_n(N)) return fail(KG_ENOTSUP, "N must be one of 16, 32, 64, 128, 256, 512");
    if (!(L > 0.0) || !std::isfinite(L)) return fail(KG_EINVAL, "L must be finite and > 0");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(KG_EINVAL, "dt must be finite and > 0");
    if (!launcher(g_opt.precision)) return fail(KG_EINVAL, "unknown precision");
    return KG_OK;
}

// release one allocation of a context (the small per-grid tables on reuse)
void release(Ctx* c, void* p, size_t bytes) {
    if (!p) return;
    for (auto it = c->allocs.begin(); it != c->allocs.end(); ++it)
        if (*it == p) {
            c->allocs.erase(it);
            cudaFree(p);
            c->bytes -= bytes;
            return;
        }
}

// A new run on the grid, precision and field kind of the current context keeps its
// device buffers (several GB at 512^3, whose release and allocation cost more than the
// set-up itself); only the tables, which depend on L and dt, and the captured step
// graph, whose launch parameters depend on them, are rebuilt.
int reuse_ctx(Ctx* c, double L, double dt, Ctx** out) {
    cudaStream_t st = stream_of(c);
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(KG_ECUDA, "reuse: stream sync");
    if (c->step_graph) cudaGraphExecDestroy(c->step_graph);
    if (c->xy_graph) cudaGraphExecDestroy(c->xy_graph);
    c->step_graph = nullptr;
    c->xy_graph = nullptr;
    c->launched = 0;
    c->plain_done = false;
    c->x_ahead = false;
    c->e_level = -1;
    const int N = c->N;
    const int m2max = 3 * (N / 2) * (N / 2);
    if (c->tw != (void*)c->tw64) release(c, c->tw, c->pl->store_bytes * N);
    release(c, c->tw64, sizeof(double2) * N);
    release(c, c->coef, sizeof(double2) * (m2max + 1));
    release(c, c->w2, sizeof(double) * (m2max + 1));
    if (c->kick) release(c, c->kick, sizeof(double2) * 3 * (m2max + 1));
    c->tw = c->tw64 = nullptr;
    c->coef = nullptr;
    c->w2 = nullptr;
    c->kick = nullptr;
    c->L = L;
    c->dt = dt;
    c->lam = g_opt.nonlinearity;
    c->have_E0 = false;
    c->E0 = 0.0;
    int rc = upload_tables(c);
    if (rc) {
        destroy(c);
        return rc;
    }
    *out = c;
    return KG_OK;
}

// a context for an N^3 run in the current options, with every buffer a step needs;
// replaces the previous context (reusing its buffers when the shapes match).  On
// failure nothing is kept.
int create_ctx(int N, double L, double dt, bool cplx, Ctx** out) {
    if (g_ctx && g_ctx->N == N && g_ctx->cplx == cplx && g_ctx->prec == g_opt.precision &&
        !std::getenv("KG_TEST_FAIL_ALLOC")) {
        Ctx* c = g_ctx;
        g_ctx = nullptr;
        return reuse_ctx(c, L, dt, out);
    }
    if (g_ctx) {
        destroy(g_ctx);
        g_ctx = nullptr;
    }
    g_alloc_counter = 0;
    Ctx* c = new Ctx();
    c->N = N;
    c->NH = N / 2 + 1;
    c->L = L;
    c->dt = dt;
    c->lam = g_opt.nonlinearity;
    c->prec = g_opt.precision;
    c->pl = launcher(c->prec);
    c->cplx = cplx;
    c->nspec = (size_t)N * N * (cplx ? N : c->NH);
    c->nphys = (size_t)N * N * N * (cplx ? 2 : 1);   // doubles of one physical field
    int rc = KG_OK;
#define KG_TRY(x)              \
    do {                       \
        rc = (x);              \
        if (rc) {              \
            destroy(c);        \
            return rc;         \
        }                      \
    } while (0)
    {
        cudaError_t e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) KG_TRY(fail(KG_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e)));
    }
    KG_TRY(dalloc(c, (void**)&c->S0, sizeof(double2) * c->nspec, "state S0"));
    KG_TRY(dalloc(c, (void**)&c->S1, sizeof(double2) * c->nspec, "state S1"));
    KG_TRY(dalloc(c, &c->W, c->pl->store_bytes * c->nspec, "work array W"));
    KG_TRY(dalloc(c, (void**)&c->dev, sizeof(KgDev), "device state"));
    if (cplx) {
        c->nparts = std::max(std::max(c->pl->xc_parts(N), c->pl->updatec_parts(N)), xc_inverse_parts(N));
    } else {
        if (c->pl->x_parts(N) <= 0) KG_TRY(fail(KG_ECUDA, "x pass occupancy query failed"));
        c->nparts = std::max(std::max(c->pl->x_parts(N), c->pl->update_parts(N)), x_inverse_parts(N));
    }
    c->nparts = std::max(c->nparts, kStrideCtas);   // the on-demand Q partials
    KG_TRY(dalloc(c, (void**)&c->part_sum, sizeof(double) * c->nparts, "partials"));
    KG_TRY(dalloc(c, (void**)&c->part_max, sizeof(double) * c->nparts, "partials max"));
    KG_TRY(dalloc(c, (void**)&c->part2, sizeof(double) * (c->nparts / 1024 + 1), "second-stage partials"));
    KG_TRY(dalloc(c, (void**)&c->scal, sizeof(double) * 8, "scalars"));
    KG_TRY(upload_tables(c));
    KG_TRY(ensure_scratch(c));
    for (auto& e : c->ev) {
        cudaError_t ee = cudaEventCreate(&e);
        if (ee != cudaSuccess) KG_TRY(fail(KG_ECUDA, "cudaEventCreate failed"));
    }
#undef KG_TRY
    *out = c;
    return KG_OK;
}

KgDev fresh_dev() {
    KgDev d;
    std::memset(&d, 0, sizeof(d));
    d.level = 0;
    d.phase = 0;
    d.frozen = 0;
    d.blowup_level = -1;
    d.energy_every = g_opt.energy_every;
    d.threshold = g_opt.blowup_threshold;
    d.P_last_level = -1000;
    d.Q_last_level = -1000;
    return d;
}

int init_common(int N, double L, double dt, const double* u0, const double* v0, bool device_ptrs) {
    int rc = check_grid(N, L, dt);
    if (rc) return rc;
    if (!u0) return fail(KG_EINVAL, "u0 is NULL");
    if (g_scheme == KG_SCHEME_COMPOSED4 && (g_opt.energy_every != 0 || g_opt.drift_tol != 0.0))
        return fail(KG_EINVAL, "energy recording and drift_tol are not defined for the composed scheme");
    const size_t n3 = (size_t)N * N * N;
    if (!device_ptrs) {
        rc = check_finite(u0, n3, "u0");
        if (!rc && v0) rc = check_finite(v0, n3, "v0");
        if (rc) return rc;
    }
    Ctx* c = nullptr;
    rc = create_ctx(N, L, dt, false, &c);
    if (rc) return rc;
#define KG_TRY(x)              \
    do {                       \
        rc = (x);              \
        if (rc) {              \
            destroy(c);        \
            return rc;         \
        }                      \
    } while (0)
    cudaStream_t st = stream_of(c);
    {
        cudaError_t e = cudaMemcpyAsync(c->phys, u0, sizeof(double) * n3,
                                        device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) KG_TRY(fail(KG_ECUDA, std::string("copy u0: ") + cudaGetErrorString(e)));
    }
    // the set-up transforms run in the pass precision where it has them (double-float), with
    // W as their work array; F^0 = R2C(lam u0^3) waits in the FP64 scratch
    Tables tb{c->tw, c->tw64, c->coef, c->w2};
    c->scheme = g_scheme;
    KG_TRY(init_state(N, c->prec, dt, c->lam, tb, c->phys, v0, device_ptrs, c->S0, c->S1, c->W, c->tmp, st,
                      c->scheme == KG_SCHEME_COMPOSED4 ? c->kick : nullptr, true));
    KgDev d = fresh_dev();
    d.scheme = c->scheme;
    if (cudaMemcpyAsync(c->dev, &d, sizeof(d), cudaMemcpyHostToDevice, st) != cudaSuccess) KG_TRY(fail(KG_ECUDA, "dev upload"));
    {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) KG_TRY(fail(KG_ECUDA, std::string("init: ") + cudaGetErrorString(e)));
    }
#undef KG_TRY
    g_ctx = c;
    return KG_OK;
}

// complex field: u0, v0 are N^3 complex values (2 N^3 doubles, interleaved re/im)
int init_common_c(int N, double L, double dt, const double* u0, const double* v0, bool device_ptrs) {
    int rc = check_grid(N, L, dt);
    if (rc) return rc;
    if (!u0) return fail(KG_EINVAL, "u0 is NULL");
    if (g_scheme != KG_SCHEME_EQ2) return fail(KG_ENOTSUP, "the composed scheme is built for real fields");
    const size_t n3 = (size_t)N * N * N;
    if (!device_ptrs) {
        rc = check_finite(u0, 2 * n3, "u0");
        if (!rc && v0) rc = check_finite(v0, 2 * n3, "v0");
        if (rc) return rc;
    }
    Ctx* c = nullptr;
    rc = create_ctx(N, L, dt, true, &c);
    if (rc) return rc;
    cudaStream_t st = stream_of(c);
    cudaError_t e = cudaMemcpyAsync(c->phys, u0, sizeof(double2) * n3,
                                    device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        destroy(c);
        return fail(KG_ECUDA, std::string("copy u0: ") + cudaGetErrorString(e));
    }
    // F^0 = FFT(lam |u0|^2 u0) waits in the FP64 scratch
    Tables tb{c->tw, c->tw64, c->coef, c->w2};
    rc = init_state_c(N, c->prec, dt, c->lam, tb, (double2*)c->phys, (const double2*)v0, device_ptrs, c->S0, c->S1,
                      c->W, c->tmp, st, true);
    KgDev d = fresh_dev();
    d.complex_field = 1;
    if (!rc && cudaMemcpyAsync(c->dev, &d, sizeof(d), cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = fail(KG_ECUDA, "dev upload");
    if (!rc) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = fail(KG_ECUDA, std::string("init: ") + cudaGetErrorString(e));
    }
    if (rc) {
        destroy(c);
        return rc;
    }
    g_ctx = c;
    return KG_OK;
}

// one step; with timed, CUDA events split it into six kernel groups and ms[0..5]
// accumulate their device times: x pass (+ its finaliser), forward y, forward z, update
// (+ its finaliser), inverse z, inverse y.
// xy = 1 or 2: the fused form (use_xy), whose first kernel runs the x pass and the forward
// y transforms of every z-plane (after their inverse y transforms when xy = 2, i.e. on
// every step of a kg_step call but its first); it ends with the z pass and leaves W
// y-forward, so the caller ends the call with one inverse y pass (xy_close).  Its time
// goes to the x slot; the forward and inverse y slots stay empty.
// skip_x: the x pass (and its finaliser) already ran for this step (kg_energy ran it ahead).
int launch_step(Ctx* c, cudaStream_t st, bool timed, float* ms, int xy = 0, bool skip_x = false) {
    const int N = c->N, NH = c->NH;
    const double h = c->L / N;
    const double p_norm = c->lam * h * h * h / 4.0;
    const double q_norm = h * h * h * inv_n3(N);
    // column geometry: NX columns per plane (N/2 + 1, or N for a complex field)
    const int NX = c->cplx ? N : NH;
    const size_t yps = (size_t)N * NX, zrs = (size_t)N * NX;
    auto col = c->cplx ? c->pl->colc : c->pl->col;
    if (timed) KG_CK(cudaEventRecord(c->ev[0], st));
    if (skip_x) {
        // W already holds the x pass's output for this step; its max |u| becomes the step's
        // (k_fin_x kept it in maxabs_peek; a frozen state keeps its value, as k_fin_x would)
        char* d = reinterpret_cast<char*>(c->dev);
        KG_CK(cudaMemcpyAsync(d + offsetof(KgDev, maxabs_last), d + offsetof(KgDev, maxabs_peek), sizeof(double),
                              cudaMemcpyDeviceToDevice, st));
    } else if (xy) {
        // (inverse y,) x pass, forward y of every z-plane in one cluster launch
        KG_CK(c->pl->xy_fused(N, xy == 2, c->W, c->dev, c->part_sum, c->part_max, c->tw, inv_n3(N), c->lam, st));
        KG_CK(launch_fin_x(c->part_sum, c->part_max, c->pl->xy_parts(N), c->dev, p_norm, st));
    } else if (c->cplx) {
        KG_CK(c->pl->passc_x(N, MODE_STEP, c->W, c->dev, c->part_sum, c->part_max, c->tw, inv_n3(N), c->lam, st));
        KG_CK(launch_fin_x(c->part_sum, c->part_max, c->pl->xc_parts(N), c->dev, p_norm, st));
    } else {
        KG_CK(c->pl->pass_x(N, MODE_STEP, c->W, c->dev, c->part_sum, c->part_max, c->tw, inv_n3(N), c->lam, st));
        KG_CK(launch_fin_x(c->part_sum, c->part_max, c->pl->x_parts(N), c->dev, p_norm, st));
    }
    if (timed) KG_CK(cudaEventRecord(c->ev[1], st));
    if (!xy) KG_CK(col(N, -1, c->W, yps, NX, N, c->tw, st));                      // forward y
    if (timed) KG_CK(cudaEventRecord(c->ev[2], st));
    const bool fused = c->pl->zstep != nullptr;
    const C4Args c4{c->kick, 3 * (N / 2) * (N / 2) + 1, {c->c4h[0], c->c4h[1], c->c4h[2]}};
    const C4Args* c4p = c->scheme == KG_SCHEME_COMPOSED4 ? &c4 : nullptr;
    if (fused) {
        // z pass: forward z FFT -> F^n, the update, inverse z FFT, in one kernel
        KG_CK(c->pl->zstep(N, c->cplx, c->W, c->S0, c->S1, c->dev, c->part_sum, c->tw, c->coef, c->w2, 1.0 / c->dt,
                           c4p, st));
        KG_CK(launch_fin_z(c->part_sum, c->pl->zstep_parts(N, c->cplx), c->part2, c->dev, q_norm, st));
    } else {
        // the IEEE FP64 passes, bound by the FP64 pipe throughout, keep the three kernels
        // (the fused form measured slower there)
        KG_CK(col(N, -1, c->W, NX, zrs, N, c->tw, st));                           // forward z -> F^n
        if (timed) KG_CK(cudaEventRecord(c->ev[3], st));
        if (c->cplx) {
            KG_CK(c->pl->updatec(N, c->W, c->S0, c->S1, c->dev, c->part_sum, c->coef, c->w2, 1.0 / c->dt, st));
            KG_CK(launch_fin_z(c->part_sum, c->pl->updatec_parts(N), c->part2, c->dev, q_norm, st));
        } else {
            KG_CK(c->pl->update(N, c->W, c->S0, c->S1, c->dev, c->part_sum, c->coef, c->w2, 1.0 / c->dt, c4p,
                                st));
            KG_CK(launch_fin_z(c->part_sum, c->pl->update_parts(N), c->part2, c->dev, q_norm, st));
        }
        if (timed) KG_CK(cudaEventRecord(c->ev[4], st));
        KG_CK(col(N, +1, c->W, NX, zrs, N, c->tw, st));                           // inverse z
    }
    if (timed) KG_CK(cudaEventRecord(c->ev[5], st));
    if (!xy) KG_CK(col(N, +1, c->W, yps, NX, N, c->tw, st));                      // inverse y
    if (timed) {
        KG_CK(cudaEventRecord(c->ev[6], st));
        KG_CK(cudaEventSynchronize(c->ev[6]));
        // segments x, forward y, (forward z, update, inverse z | fused z pass), inverse y;
        // a fused z pass is reported in ms[2] and leaves ms[3], ms[4] at zero
        const int split[6][3] = {{0, 1, 0}, {1, 2, 1}, {2, 3, 2}, {3, 4, 3}, {4, 5, 4}, {5, 6, 5}};
        const int joint[4][3] = {{0, 1, 0}, {1, 2, 1}, {2, 5, 2}, {5, 6, 5}};
        const int count = fused ? 4 : 6;
        for (int g = 0; g < count; g++) {
            const int* sg = fused ? joint[g] : split[g];
            float t = 0.f;
            KG_CK(cudaEventElapsedTime(&t, c->ev[sg[0]], c->ev[sg[1]]));
            ms[sg[2]] += t;
        }
    }
    return KG_OK;
}

// capture one step (its launches) into a graph; every decision of a step is made
// on the device from KgDev, so the same graph serves every later step
int ensure_step_graph(Ctx* c, cudaStream_t st) {
    if (c->step_graph) return KG_OK;
    cudaGraph_t g = nullptr;
    KG_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = launch_step(c, st, false, nullptr);
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return rc ? rc : fail(KG_ECUDA, std::string("step graph capture: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&c->step_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(KG_ECUDA, std::string("step graph instantiate: ") + cudaGetErrorString(e));
    return KG_OK;
}

// the fused xy form serves the FP32 passes of a real field under Eq. (2) from N = 64 on,
// when kg_set_xy_fusion asked for it
bool use_xy(const Ctx* c) {
    return g_xy_fusion && c->pl->xy_fused && c->pl->xy_parts && !c->cplx && c->scheme == KG_SCHEME_EQ2 && c->N >= 64 &&
           c->pl->xy_parts(c->N) > 0;
}

// the inverse y pass that ends a kg_step call of the fused form (W back to the y-inverse)
int xy_close(Ctx* c, cudaStream_t st, bool timed, float* ms) {
    const int N = c->N, NX = c->NH;
    if (timed) KG_CK(cudaEventRecord(c->ev[5], st));
    KG_CK(c->pl->col(N, +1, c->W, (size_t)N * NX, NX, N, c->tw, st));
    if (timed) {
        KG_CK(cudaEventRecord(c->ev[6], st));
        KG_CK(cudaEventSynchronize(c->ev[6]));
        float t = 0.f;
        KG_CK(cudaEventElapsedTime(&t, c->ev[5], c->ev[6]));
        ms[5] += t;
    }
    return KG_OK;
}

// capture one step of the fused form with its inverse y transforms
int ensure_xy_graph(Ctx* c, cudaStream_t st) {
    if (c->xy_graph) return KG_OK;
    cudaGraph_t g = nullptr;
    KG_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = launch_step(c, st, false, nullptr, 2);
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return rc ? rc : fail(KG_ECUDA, std::string("xy step graph capture: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&c->xy_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(KG_ECUDA, std::string("xy step graph instantiate: ") + cudaGetErrorString(e));
    return KG_OK;
}

int read_dev(Ctx* c, KgDev* d) {
    cudaStream_t st = stream_of(c);
    KG_CK(cudaMemcpyAsync(d, c->dev, sizeof(KgDev), cudaMemcpyDeviceToHost, st));
    KG_CK(cudaStreamSynchronize(st));
    return KG_OK;
}

// P of the FP64 state array that is current (older = false) or previous (older = true)
int p_from_state(Ctx* c, bool older, double* out) {
    const int N = c->N;
    const double h = c->L / N;
    cudaStream_t st = stream_of(c);
    // phase 0: S0 current; the "older" array is the other one
    int rc = older ? inverse_yz_f64(c, c->S1, c->S0, c->dev) : inverse_yz_f64(c, c->S0, c->S1, c->dev);
    if (rc) return rc;
    if (c->cplx) {
        KG_CK(launch_xc_inverse(N, c->tmp, nullptr, c->tw64, inv_n3(N), c->part_sum, st));
        KG_CK(launch_fin_sum(c->part_sum, xc_inverse_parts(N), c->lam * h * h * h / 4.0, c->scal, st));
    } else {
        KG_CK(launch_x_inverse(N, c->tmp, nullptr, c->tw64, inv_n3(N), c->part_sum, st));
        KG_CK(launch_fin_sum(c->part_sum, x_inverse_parts(N), c->lam * h * h * h / 4.0, c->scal, st));
    }
    KG_CK(cudaMemcpyAsync(out, c->scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    KG_CK(cudaStreamSynchronize(st));
    return KG_OK;
}

}  // namespace

namespace kg {
// lets other translation units of the library report through kg_last_error()
int set_last_error(int code, const std::string& msg) { return fail(code, msg); }
const char* ens_tune_cache();   // kg_ensemble.cu
}  // namespace kg

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int kg_init(int N, double L, double dt, const double* u0, const double* v0) {
    return init_common(N, L, dt, u0, v0, false);
}

int kg_init_device(int N, double L, double dt, const double* d_u0, const double* d_v0) {
    return init_common(N, L, dt, d_u0, d_v0, true);
}

// Energy of the composed scheme at the current (integer) step, in FP64: the continuous
// functional of section 1.1 with the synchronised velocity p (the stored P plus the
// pending half kick), E = (h^3/N^3) sum_k w_k (|p|^2 + omega^2 |uh|^2)/2 - lam (h^3/4) sum u^4
int energy_composed(Ctx* c, double* E) {
    const int N = c->N;
    const double h = c->L / N;
    cudaStream_t st = stream_of(c);
    int rc = inverse_yz_f64(c, c->S0, c->S1, c->dev);            // phase 0: S0 = uh, S1 = P
    if (rc) return rc;
    KG_CK(launch_x_inverse(N, c->tmp, c->phys, c->tw64, inv_n3(N), c->part_sum, st));   // u^n, sum u^4
    KG_CK(launch_fin_sum(c->part_sum, x_inverse_parts(N), c->lam * h * h * h / 4.0, c->scal + 1, st));
    rc = forward3d_f64(N, c->phys, c->tmp, c->tw64, 1, c->lam, st);   // F = R2C(lam u^3)
    if (rc) return rc;
    KG_CK(launch_energy_c4(N, c->S0, c->S1, c->tmp, c->kick, c->w2, c->part_sum, kStrideCtas, st));
    KG_CK(launch_fin_sum(c->part_sum, kStrideCtas, h * h * h * inv_n3(N), c->scal, st));
    double v[2];
    KG_CK(cudaMemcpyAsync(v, c->scal, sizeof(v), cudaMemcpyDeviceToHost, st));
    KG_CK(cudaStreamSynchronize(st));
    *E = v[0] - v[1];
    return KG_OK;
}

// pipeline passes of one step: one, or three substeps for the composed scheme
int passes_per_step(const Ctx* c) { return c->scheme == KG_SCHEME_COMPOSED4 ? 3 : 1; }

int kg_step(int n) {
    Ctx* c = g_ctx;
    if (!c) return fail(KG_ESTATE, "kg_step before kg_init");
    if (n < 0) return fail(KG_EINVAL, "n < 0");
    cudaStream_t st = stream_of(c);
    long long passes = (long long)n * passes_per_step(c);
    if (c->x_ahead && passes > 0) {
        // the first step's x pass ran in kg_energy: the rest of that step, outside the graphs
        c->x_ahead = false;
        const int rc = launch_step(c, st, false, nullptr, 0, true);
        if (rc) return rc;
        c->launched++;
        passes--;
    }
    if (use_xy(c) && passes > 0) {
        // first step without the inverse y transforms (W holds the y-inverse between
        // calls), the others from the captured fused step, then one inverse y pass
        for (long long i = 0; i < passes; i++) {
            int rc;
            if (i == 0) {
                rc = launch_step(c, st, false, nullptr, 1);
            } else {
                rc = ensure_xy_graph(c, st);
                if (!rc && cudaGraphLaunch(c->xy_graph, st) != cudaSuccess) rc = fail(KG_ECUDA, "cudaGraphLaunch(xy)");
            }
            if (rc) return rc;
            c->launched++;
        }
        return xy_close(c, st, false, nullptr);
    }
    for (long long i = 0; i < passes; i++) {
        int rc;
        if (!c->plain_done) {
            rc = launch_step(c, st, false, nullptr);   // first step direct: it also sets kernel attributes
            c->plain_done = true;
        } else {
            rc = ensure_step_graph(c, st);
            if (!rc && cudaGraphLaunch(c->step_graph, st) != cudaSuccess) rc = fail(KG_ECUDA, "cudaGraphLaunch(step)");
        }
        if (rc) return rc;
        c->launched++;
    }
    return KG_OK;
}

int kg_step_timed(int n, float* ms) {
    Ctx* c = g_ctx;
    if (!c) return fail(KG_ESTATE, "kg_step_timed before kg_init");
    if (n < 0 || !ms) return fail(KG_EINVAL, "bad arguments");
    for (int p = 0; p < 6; p++) ms[p] = 0.f;
    cudaStream_t st = stream_of(c);
    long long passes = (long long)n * passes_per_step(c);
    if (c->x_ahead && passes > 0) {
        c->x_ahead = false;
        const int rc = launch_step(c, st, true, ms, 0, true);
        if (rc) return rc;
        c->launched++;
        passes--;
    }
    const bool xy = use_xy(c);
    for (long long i = 0; i < passes; i++) {
        int rc = launch_step(c, st, true, ms, xy ? (i == 0 ? 1 : 2) : 0);
        if (rc) return rc;
        c->launched++;
    }
    if (xy && passes > 0) return xy_close(c, st, true, ms);
    return KG_OK;
}

int kg_energy(double* E) {
    Ctx* c = g_ctx;
    if (!c) return fail(KG_ESTATE, "kg_energy before kg_init");
    if (!E) return fail(KG_EINVAL, "E is NULL");
    if (c->scheme == KG_SCHEME_COMPOSED4) return energy_composed(c, E);
    const int N = c->N;
    const double h = c->L / N;
    cudaStream_t st = stream_of(c);
    KgDev d;
    int rc = read_dev(c, &d);
    if (rc) return rc;
    const long long n = d.level;
    double Q, Pm, Pn;
    if (c->e_level == n) {
        // asked again at the same level (after an x pass run ahead W no longer holds u^n's
        // transform to peek at): the value computed then
        *E = c->e_value;
        if (g_opt.drift_tol > 0.0 && c->have_E0 && std::fabs(*E - c->E0) > g_opt.drift_tol * std::fabs(c->E0))
            return fail(KG_EDRIFT, "energy drift beyond drift_tol");
        return KG_OK;
    }
    // Q^{n-1/2}
    if (d.Q_last_level == n - 1) {
        Q = d.Q_last;
    } else {
        const double2* cur = d.phase ? c->S1 : c->S0;
        const double2* old = d.phase ? c->S0 : c->S1;
        const int np = kStrideCtas;
        KG_CK(launch_energy_q(N, cur, old, c->w2, 1.0 / c->dt, c->part_sum, np, c->cplx, st));
        KG_CK(launch_fin_sum(c->part_sum, np, h * h * h * inv_n3(N), c->scal, st));
        KG_CK(cudaMemcpyAsync(&Q, c->scal, sizeof(double), cudaMemcpyDeviceToHost, st));
        KG_CK(cudaStreamSynchronize(st));
    }
    // P^{n-1}
    if (d.P_last_level == n - 1) {
        Pm = d.P_last;
    } else {
        rc = p_from_state(c, true, &Pm);
        if (rc) return rc;
    }
    // P^n: from W (which holds the yz-inverse of uh^n) unless the state froze.  For a real
    // field stepped by separate passes, the next step's x pass runs now with P^n recorded
    // (it forms u^n anyway) and kg_step skips it; otherwise a read-only peek pass.
    if (!d.frozen && !c->cplx && !use_xy(c) && !c->x_ahead) {
        const int one = 1;
        KG_CK(cudaMemcpyAsync(reinterpret_cast<char*>(c->dev) + offsetof(KgDev, record_p), &one, sizeof(int),
                              cudaMemcpyHostToDevice, st));
        KG_CK(c->pl->pass_x(N, MODE_STEP, c->W, c->dev, c->part_sum, c->part_max, c->tw, inv_n3(N), c->lam, st));
        KG_CK(launch_fin_x(c->part_sum, c->part_max, c->pl->x_parts(N), c->dev, c->lam * h * h * h / 4.0, st));
        c->x_ahead = true;
        KgDev d2;
        rc = read_dev(c, &d2);
        if (rc) return rc;
        if (d2.P_last_level != n) return fail(KG_ECUDA, "kg_energy: the x pass run ahead recorded no P");
        Pn = d2.P_last;
    } else if (!d.frozen) {
        if (c->cplx) {
            KG_CK(c->pl->passc_x(N, MODE_PEEK, c->W, c->dev, c->part_sum, c->part_max, c->tw, inv_n3(N), c->lam,
                                 st));
            KG_CK(launch_fin_peek(c->part_sum, c->part_max, c->pl->xc_parts(N), c->dev, c->lam * h * h * h / 4.0,
                                  st));
        } else {
            KG_CK(c->pl->pass_x(N, MODE_PEEK, c->W, c->dev, c->part_sum, c->part_max, c->tw, inv_n3(N), c->lam,
                                st));
            KG_CK(launch_fin_peek(c->part_sum, c->part_max, c->pl->x_parts(N), c->dev, c->lam * h * h * h / 4.0,
                                  st));
        }
        KgDev d2;
        rc = read_dev(c, &d2);
        if (rc) return rc;
        Pn = d2.P_peek;
    } else {
        rc = p_from_state(c, false, &Pn);
        if (rc) return rc;
    }
    *E = Q - 0.5 * (Pm + Pn);
    c->e_level = n;
    c->e_value = *E;
    if (!c->have_E0) {
        c->have_E0 = true;
        c->E0 = *E;
    } else if (g_opt.drift_tol > 0.0 && std::fabs(*E - c->E0) > g_opt.drift_tol * std::fabs(c->E0)) {
        return fail(KG_EDRIFT, "energy drift beyond drift_tol");
    }
    return KG_OK;
}

int kg_fetch_device(double* d_u) {
    Ctx* c = g_ctx;
    if (!c) return fail(KG_ESTATE, "kg_fetch before kg_init");
    if (!d_u) return fail(KG_EINVAL, "output pointer is NULL");
    if (c->cplx) return fail(KG_ESTATE, "the context holds a complex field: use kg_fetch_complex");
    if (c->pl->x_readout) {
        // read-out in the pass precision (double-float): inverse z and y of uh^n into the FP64
        // scratch used as a W-format array, then the inverse x into d_u
        const int N = c->N, NH = c->NH;
        cudaStream_t st = stream_of(c);
        KG_CK(c->pl->col_from_f64(N, c->S0, c->S1, c->dev, c->tmp, NH, (size_t)N * NH, N, c->tw, st));
        KG_CK(c->pl->col(N, +1, c->tmp, (size_t)N * NH, NH, N, c->tw, st));
        KG_CK(c->pl->x_readout(N, c->tmp, d_u, c->tw, inv_n3(N), st));
        return KG_OK;
    }
    int rc = inverse_yz_f64(c, c->S0, c->S1, c->dev);
    if (rc) return rc;
    KG_CK(launch_x_inverse(c->N, c->tmp, d_u, c->tw64, inv_n3(c->N), nullptr, stream_of(c)));
    return KG_OK;
}

int kg_fetch(double* u) {
    Ctx* c = g_ctx;
    if (!c) return fail(KG_ESTATE, "kg_fetch before kg_init");
    if (!u) return fail(KG_EINVAL, "output pointer is NULL");
    if (c->cplx) return fail(KG_ESTATE, "the context holds a complex field: use kg_fetch_complex");
    int rc = kg_fetch_device(c->phys);
    if (rc) return rc;
    cudaStream_t st = stream_of(c);
    KG_CK(cudaMemcpyAsync(u, c->phys, sizeof(double) * c->nphys, cudaMemcpyDeviceToHost, st));
    KG_CK(cudaStreamSynchronize(st));
    return KG_OK;
}

int kg_init_complex(int N, double L, double dt, const double* u0, const double* v0) {
    return init_common_c(N, L, dt, u0, v0, false);
}

int kg_init_complex_device(int N, double L, double dt, const double* d_u0, const double* d_v0) {
    return init_common_c(N, L, dt, d_u0, d_v0, true);
}

int kg_fetch_complex_device(double* d_u) {
    Ctx* c = g_ctx;
    if (!c) return fail(KG_ESTATE, "kg_fetch_complex before kg_init_complex");
    if (!d_u) return fail(KG_EINVAL, "output pointer is NULL");
    if (!c->cplx) return fail(KG_ESTATE, "the context holds a real field: use kg_fetch");
    if (c->pl->xc_readout) {
        // read-out in the pass precision (double-float), as kg_fetch_device
        const int N = c->N;
        cudaStream_t st = stream_of(c);
        KG_CK(c->pl->colc_from_f64(N, c->S0, c->S1, c->dev, c->tmp, N, (size_t)N * N, N, c->tw, st));
        KG_CK(c->pl->colc(N, +1, c->tmp, (size_t)N * N, N, N, c->tw, st));
        KG_CK(c->pl->xc_readout(N, c->tmp, (double2*)d_u, c->tw, inv_n3(N), st));
        return KG_OK;
    }
    int rc = inverse_yz_f64(c, c->S0, c->S1, c->dev);
    if (rc) return rc;
    KG_CK(launch_xc_inverse(c->N, c->tmp, (double2*)d_u, c->tw64, inv_n3(c->N), nullptr, stream_of(c)));
    return KG_OK;
}

int kg_fetch_complex(double* u) {
    Ctx* c = g_ctx;
    if (!c) return fail(KG_ESTATE, "kg_fetch_complex before kg_init_complex");
    if (!u) return fail(KG_EINVAL, "output pointer is NULL");
    if (!c->cplx) return fail(KG_ESTATE, "the context holds a real field: use kg_fetch");
    int rc = kg_fetch_complex_device(c->phys);
    if (rc) return rc;
    cudaStream_t st = stream_of(c);
    KG_CK(cudaMemcpyAsync(u, c->phys, sizeof(double) * c->nphys, cudaMemcpyDeviceToHost, st));
    KG_CK(cudaStreamSynchronize(st));
    return KG_OK;
}

int kg_fetch_spectral(double* a, double* b) {
    Ctx* c = g_ctx;
    if (!c) return fail(KG_ESTATE, "kg_fetch_spectral before kg_init");
    KgDev d;
    int rc = read_dev(c, &d);
    if (rc) return rc;
    const double2* cur = d.phase ? c->S1 : c->S0;
    const double2* old = d.phase ? c->S0 : c->S1;
    if (a) KG_CK(cudaMemcpy(a, cur, sizeof(double2) * c->nspec, cudaMemcpyDeviceToHost));
    if (b) KG_CK(cudaMemcpy(b, old, sizeof(double2) * c->nspec, cudaMemcpyDeviceToHost));
    return KG_OK;
}

int kg_status(long long* level, int* frozen, long long* blowup_level, double* maxabs) {
    Ctx* c = g_ctx;
    if (!c) return fail(KG_ESTATE, "kg_status before kg_init");
    KgDev d;
    int rc = read_dev(c, &d);
    if (rc) return rc;
    if (level) *level = d.level;
    if (frozen) *frozen = d.frozen;
    if (blowup_level) *blowup_level = d.blowup_level;
    if (maxabs) *maxabs = d.maxabs_last;
    return KG_OK;
}

int kg_finalize(void) {
    if (g_ctx) {
        destroy(g_ctx);
        g_ctx = nullptr;
    }
    return KG_OK;
}

int kg_set_stream(void* stream) {
    if (g_ctx && g_user_stream != (cudaStream_t)stream) {
        // order the switch: work already queued on the old stream completes first
        cudaStream_t old = stream_of(g_ctx);
        KG_CK(cudaStreamSynchronize(old));
    }
    g_user_stream = (cudaStream_t)stream;
    return KG_OK;
}

int kg_set_options(const kg_options* o) {
    if (!o) return fail(KG_EINVAL, "options pointer is NULL");
    if (!launcher(o->precision)) return fail(KG_EINVAL, "unknown precision");
    if (o->energy_every < 0) return fail(KG_EINVAL, "energy_every < 0");
    if (!std::isfinite(o->nonlinearity) || !std::isfinite(o->blowup_threshold) || !std::isfinite(o->drift_tol))
        return fail(KG_EINVAL, "non-finite option");
    if (o->tune_cache) kg_ens_set_tune_cache(o->tune_cache);   // copied; NULL leaves it as set
    g_opt = *o;
    g_opt.tune_cache = nullptr;   // kg_get_options reports the library's own copy
    if (g_ctx) {
        // energy cadence and blow-up threshold apply at once; lam and precision at the next init
        Ctx* c = g_ctx;
        KgDev d;
        int rc = read_dev(c, &d);
        if (rc) return rc;
        d.energy_every = o->energy_every;
        d.threshold = o->blowup_threshold;
        cudaStream_t st = stream_of(c);
        KG_CK(cudaMemcpyAsync(c->dev, &d, sizeof(d), cudaMemcpyHostToDevice, st));
        KG_CK(cudaStreamSynchronize(st));
    }
    return KG_OK;
}

int kg_get_options(kg_options* o) {
    if (!o) return fail(KG_EINVAL, "options pointer is NULL");
    *o = g_opt;
    o->tune_cache = kg::ens_tune_cache();
    return KG_OK;
}

int kg_set_scheme(int scheme) {
    if (scheme != KG_SCHEME_EQ2 && scheme != KG_SCHEME_COMPOSED4) return fail(KG_EINVAL, "unknown scheme");
    g_scheme = scheme;
    return KG_OK;
}

int kg_set_xy_fusion(int on) {
    if (on != 0 && on != 1) return fail(KG_EINVAL, "kg_set_xy_fusion: on must be 0 or 1");
    if (g_ctx && g_xy_fusion != on) {
        // the next kg_step takes the other form; W holds the y-inverse between calls in both
        cudaStream_t st = stream_of(g_ctx);
        KG_CK(cudaStreamSynchronize(st));
    }
    g_xy_fusion = on;
    return KG_OK;
}

int kg_get_xy_fusion(int* on, int* active) {
    if (!on) return fail(KG_EINVAL, "kg_get_xy_fusion: NULL");
    *on = g_xy_fusion;
    if (active) *active = (g_ctx && use_xy(g_ctx)) ? 1 : 0;
    return KG_OK;
}

int kg_get_scheme(int* scheme) {
    if (!scheme) return fail(KG_EINVAL, "scheme is NULL");
    *scheme = g_scheme;
    return KG_OK;
}

int kg_memory(size_t* bytes) {
    if (!bytes) return fail(KG_EINVAL, "NULL");
    *bytes = g_ctx ? g_ctx->bytes : 0;
    return KG_OK;
}

unsigned long long kg_state_checksum(const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    unsigned long long sum = 0;
    for (size_t i = 0; i < n / 8; i++) {
        unsigned long long w;
        std::memcpy(&w, b + 8 * i, 8);
        const unsigned r = (unsigned)(i & 63);
        sum += r ? (w << r) | (w >> (64 - r)) : w;
    }
    return sum;
}

int kg_save_state(void* h, size_t cap, size_t* used) {
    Ctx* c = g_ctx;
    if (!c) return fail(KG_ESTATE, "kg_save_state before kg_init");
    if (!used) return fail(KG_EINVAL, "used is NULL");
    const size_t arr = sizeof(double2) * c->nspec;
    const size_t need = sizeof(kg_state_header) + 2 * arr;
    *used = need;
    if (!h) return KG_OK;
    if (cap < need) return fail(KG_EINVAL, "checkpoint buffer smaller than kg_save_state(NULL) reported");
    KgDev d;
    int rc = read_dev(c, &d);
    if (rc) return rc;
    kg_state_header hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, KG_STATE_MAGIC, 8);
    hd.version = KG_STATE_VERSION;
    hd.header_bytes = (unsigned)sizeof(hd);
    hd.N = c->N;
    hd.precision = c->prec;
    hd.energy_every = d.energy_every;
    hd.frozen = d.frozen;
    hd.L = c->L;
    hd.dt = c->dt;
    hd.nonlinearity = c->lam;
    hd.blowup_threshold = d.threshold;
    hd.drift_tol = g_opt.drift_tol;
    hd.level = d.level;
    hd.blowup_level = d.blowup_level;
    hd.maxabs_last = d.maxabs_last;
    hd.P_last = d.P_last;
    hd.P_last_level = d.P_last_level;
    hd.Q_last = d.Q_last;
    hd.Q_last_level = d.Q_last_level;
    hd.have_E0 = c->have_E0 ? 1 : 0;
    hd.E0 = c->E0;
    hd.complex_field = c->cplx ? 1 : 0;
    hd.scheme = c->scheme;
    hd.payload_bytes = 2 * arr;
    unsigned char* base = (unsigned char*)h;
    cudaStream_t st = stream_of(c);
    const double2* cur = d.phase ? c->S1 : c->S0;
    const double2* old = d.phase ? c->S0 : c->S1;
    KG_CK(cudaMemcpyAsync(base + sizeof(hd), cur, arr, cudaMemcpyDeviceToHost, st));
    KG_CK(cudaMemcpyAsync(base + sizeof(hd) + arr, old, arr, cudaMemcpyDeviceToHost, st));
    KG_CK(cudaStreamSynchronize(st));
    hd.checksum = kg_state_checksum(base + sizeof(hd), 2 * arr);
    std::memcpy(base, &hd, sizeof(hd));
    return KG_OK;
}

int kg_load_state(const void* h, size_t len) {
    if (!h) return fail(KG_EINVAL, "checkpoint pointer is NULL");
    if (len < sizeof(kg_state_header)) return fail(KG_EINVAL, "checkpoint shorter than its header");
    kg_state_header hd;
    std::memcpy(&hd, h, sizeof(hd));
    if (std::memcmp(hd.magic, KG_STATE_MAGIC, 8) != 0) return fail(KG_EINVAL, "not a checkpoint (magic)");
    if (hd.version != KG_STATE_VERSION) return fail(KG_EINVAL, "unknown checkpoint version");
    if (hd.header_bytes != sizeof(hd)) return fail(KG_EINVAL, "checkpoint header size mismatch");
    if (!supported_n(hd.N)) return fail(KG_ENOTSUP, "checkpoint N not supported");
    if (!launcher(hd.precision)) return fail(KG_EINVAL, "checkpoint precision unknown");
    if (!(hd.L > 0.0) || !std::isfinite(hd.L) || !(hd.dt > 0.0) || !std::isfinite(hd.dt) ||
        !std::isfinite(hd.nonlinearity) || !std::isfinite(hd.blowup_threshold) || !std::isfinite(hd.drift_tol) ||
        hd.energy_every < 0 || hd.level < 0 || (hd.frozen != 0 && hd.frozen != 1) ||
        (hd.complex_field != 0 && hd.complex_field != 1) ||
        (hd.scheme != KG_SCHEME_EQ2 && hd.scheme != KG_SCHEME_COMPOSED4) ||
        (hd.scheme == KG_SCHEME_COMPOSED4 && (hd.complex_field != 0 || hd.energy_every != 0 || hd.drift_tol != 0.0)))
        return fail(KG_EINVAL, "checkpoint header field out of range");
    const bool cplx = hd.complex_field == 1;
    const size_t nspec = (size_t)hd.N * hd.N * (cplx ? hd.N : hd.N / 2 + 1);
    const size_t arr = sizeof(double2) * nspec;
    if (hd.payload_bytes != 2 * arr) return fail(KG_EINVAL, "checkpoint payload size does not match N");
    if (len < sizeof(hd) + 2 * arr) return fail(KG_EINVAL, "checkpoint truncated");
    const unsigned char* base = (const unsigned char*)h;
    if (kg_state_checksum(base + sizeof(hd), 2 * arr) != hd.checksum) return fail(KG_EINVAL, "checkpoint checksum mismatch");

    kg_options o = g_opt;
    o.precision = hd.precision;
    o.energy_every = hd.energy_every;
    o.nonlinearity = hd.nonlinearity;
    o.blowup_threshold = hd.blowup_threshold;
    o.drift_tol = hd.drift_tol;
    g_opt = o;
    g_scheme = hd.scheme;
    Ctx* c = nullptr;
    int rc = create_ctx(hd.N, hd.L, hd.dt, cplx, &c);
    if (rc) return rc;
    c->scheme = hd.scheme;
    const int N = c->N, NX = cplx ? N : c->NH;
    cudaStream_t st = stream_of(c);
    KgDev d = fresh_dev();
    d.level = hd.level;
    d.frozen = hd.frozen;
    d.blowup_level = hd.blowup_level;
    d.maxabs_last = hd.maxabs_last;
    d.P_last = hd.P_last;
    d.P_last_level = hd.P_last_level;
    d.Q_last = hd.Q_last;
    d.Q_last_level = hd.Q_last_level;
    d.complex_field = cplx ? 1 : 0;
    d.scheme = c->scheme;
    cudaError_t e = cudaMemcpyAsync(c->S0, base + sizeof(hd), arr, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->S1, base + sizeof(hd) + arr, arr, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->dev, &d, sizeof(d), cudaMemcpyHostToDevice, st);
    // W = the yz inverse of uh^n in the pass precision, as the last two transforms of a step leave it
    auto col = cplx ? c->pl->colc : c->pl->col;
    auto col_f64 = cplx ? c->pl->colc_from_f64 : c->pl->col_from_f64;
    if (e == cudaSuccess) e = col_f64(N, c->S0, c->S1, nullptr, c->W, NX, (size_t)N * NX, N, c->tw, st);
    if (e == cudaSuccess) e = col(N, +1, c->W, (size_t)N * NX, NX, N, c->tw, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        destroy(c);
        return fail(KG_ECUDA, std::string("kg_load_state: ") + cudaGetErrorString(e));
    }
    c->have_E0 = hd.have_E0 != 0;
    c->E0 = hd.E0;
    g_ctx = c;
    return KG_OK;
}

const char* kg_last_error(void) { return g_err.c_str(); }

}  // extern "C"
