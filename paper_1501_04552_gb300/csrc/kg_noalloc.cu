// kg_noalloc.cu -- kg_energy_q_noalloc: the quadratic energy Q of a Fourier state
// pair for callers that cannot allocate device memory.
//
// Who needs it: applications whose device memory is owned by someone else (a
// framework's caching allocator, or a fixed pool reserved at start-up under a
// hard memory budget) and loops that cannot afford the implicit device
// synchronisation of cudaMalloc/cudaFree.  They hand in device arrays they already
// own and get the result in a device scalar they already own.
//
// How: the reduction's per-CTA partial sums, which the context-based path keeps
// in a cudaMalloc'd buffer, live here in a file-scope static device array of
// kStaticParts doubles (64 KiB), allocated on each GPU when the library's device
// code is loaded there and held until the process exits.  Host code may not pass the array's name to a
// kernel (on the host it is only a stand-in symbol); its device address is taken
// with cudaGetSymbolAddress once per device, with that device current, on the
// first call made on it.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <string>

#include "../../include/kg.h"
#include "kg_fft.cuh"

using namespace kg;

namespace {

constexpr int kStaticParts = 8192;                  // partial sums the static scratch holds
constexpr long long kModesPerPart = 16384;           // modes one CTA sums
constexpr long long kMaxModes = kStaticParts * kModesPerPart;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// the shared scratch: partial sums of the last call on this device
__device__ __align__(256) double g_q_scratch[kStaticParts];

// the array's device address on each device, looked up on the first call made there.
// Several host threads may make that first call at once: each looks the address up (it is
// the same on every lookup) and stores it; the slot is atomic so that no read races a write.
std::atomic<double*> g_scratch_addr[kMaxDevices];

// Q partials: CTA b sums the weighted energy terms of modes [b M, (b+1) M), M = kModesPerPart
__global__ void __launch_bounds__(kThreads) k_energy_q_parts(const double2* __restrict__ x, const double2* __restrict__ y,
                                                             int N, long long nmodes, double kf2, double inv_dt,
                                                             double* __restrict__ parts) {
    __shared__ double red[96];
    const int NH = N / 2 + 1;
    const long long begin = (long long)blockIdx.x * kModesPerPart;
    const long long end = begin + kModesPerPart < nmodes ? begin + kModesPerPart : nmodes;
    NSum acc;
    acc.s = 0.0;
    acc.c = 0.0;
    for (long long i = begin + threadIdx.x; i < end; i += kThreads) {
        const int kx = (int)(i % NH);
        const int ky = (int)((i / NH) % N);
        const int kz = (int)(i / ((long long)NH * N));
        const int my = ky <= N / 2 ? ky : ky - N, mz = kz <= N / 2 ? kz : kz - N;
        const double om2 = 1.0 + kf2 * (double)(kx * kx + my * my + mz * mz);
        const double w = (kx == 0 || kx == N / 2) ? 1.0 : 2.0;
        const double2 a = x[i], b = y[i];
        const double dre = (a.x - b.x) * inv_dt, dim = (a.y - b.y) * inv_dt;
        const double sre = a.x + b.x, sim = a.y + b.y;
        acc.add(w * (0.5 * (dre * dre + dim * dim) + 0.125 * om2 * (sre * sre + sim * sim)));
    }
    double mx = 0.0;
    block_reduce<kThreads>(acc, mx, red);
    if (threadIdx.x == 0) parts[blockIdx.x] = acc.value();
}

__global__ void __launch_bounds__(1024) k_energy_q_total(const double* __restrict__ parts, int count, double norm,
                                                         double* __restrict__ out) {
    __shared__ double red[96];
    NSum acc;
    acc.s = 0.0;
    acc.c = 0.0;
    for (int i = threadIdx.x; i < count; i += 1024) acc.add(parts[i]);
    double mx = 0.0;
    block_reduce<1024>(acc, mx, red);
    if (threadIdx.x == 0) *out = norm * acc.value();
}

}  // namespace

namespace kg {
int set_last_error(int code, const std::string& msg);  // kg_api.cu: the text kg_last_error() returns
}

static int noalloc_fail(int code, const std::string& msg) { return kg::set_last_error(code, msg); }

extern "C" int kg_energy_q_noalloc(int N, double L, double dt, const double* d_cur, const double* d_old, double* d_Q,
                                   void* stream) {
    if (N < 2 || (N & 1)) return noalloc_fail(KG_ENOTSUP, "kg_energy_q_noalloc: N must be even and >= 2");
    const long long nmodes = (long long)N * N * (N / 2 + 1);
    if (nmodes > kMaxModes)
        return noalloc_fail(KG_ENOTSUP, "kg_energy_q_noalloc: N*N*(N/2+1) = " + std::to_string(nmodes) +
                                            " modes exceeds the static scratch maximum of " +
                                            std::to_string(kMaxModes) + " (N <= 644)");
    if (!(L > 0.0) || !std::isfinite(L) || !(dt > 0.0) || !std::isfinite(dt))
        return noalloc_fail(KG_EINVAL, "kg_energy_q_noalloc: L and dt must be finite and > 0");
    if (!d_cur || !d_old || !d_Q) return noalloc_fail(KG_EINVAL, "kg_energy_q_noalloc: NULL pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(KG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(KG_ENOTSUP, "kg_energy_q_noalloc: device index too large");
    double* parts = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!parts) {  // set-up, once per device, with that device current
        e = cudaGetSymbolAddress((void**)&parts, g_q_scratch);
        if (e != cudaSuccess || !parts)
            return noalloc_fail(KG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev].store(parts, std::memory_order_release);
    }
    const int nparts = (int)((nmodes + kModesPerPart - 1) / kModesPerPart);
    const double kf = 2.0 * 3.14159265358979323846 / L;
    const double h = L / N;
    const double norm = h * h * h / ((double)N * (double)N * (double)N);
    cudaStream_t st = (cudaStream_t)stream;
    k_energy_q_parts<<<nparts, kThreads, 0, st>>>((const double2*)d_cur, (const double2*)d_old, N, nmodes, kf * kf,
                                                 1.0 / dt, parts);
    k_energy_q_total<<<1, 1024, 0, st>>>(parts, nparts, norm, d_Q);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(KG_ECUDA, std::string("kg_energy_q_noalloc launch: ") + cudaGetErrorString(e));
    return KG_OK;
}
