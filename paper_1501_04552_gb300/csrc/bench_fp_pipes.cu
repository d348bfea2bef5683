// bench_fp_pipes.cu -- issue rates of the arithmetic the double-float transforms are built
// from, measured on the device this runs on (a standalone microbenchmark; not part of libkg).
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o /tmp/bench_fp_pipes \
//        paper_1501_04552_gb300/csrc/bench_fp_pipes.cu && /tmp/bench_fp_pipes
//
// Every kernel runs 8 CTAs of 256 threads per SM; each thread keeps 16 independent
// dependency chains (8 for the two-lane forms) so that latency is hidden and the issue
// rate or the pipe is the limit.  Reported: lane operations per second and per SM per
// clock at the SM clock the run reads back.  The last two kernels time one radix-2 layer
// of lazy double-float sums and seven twiddle products on 8 values, written with scalar
// FP32 instructions and with the packed FP32x2 forms of kg_arith.cuh.
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include "kg_arith.cuh"

using namespace kg;

#define CK(x)                                                                            \
    do {                                                                                 \
        cudaError_t e_ = (x);                                                            \
        if (e_ != cudaSuccess) {                                                         \
            printf("CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
            exit(1);                                                                     \
        }                                                                                \
    } while (0)

__device__ __forceinline__ float ffma1(float a, float b, float c) {
    float d;
    asm volatile("fma.rn.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ double dfma1(double a, double b, double c) {
    double d;
    asm volatile("fma.rn.f64 %0, %1, %2, %3;" : "=d"(d) : "d"(a), "d"(b), "d"(c));
    return d;
}
__device__ __forceinline__ double dadd1(double a, double b) {
    double d;
    asm volatile("add.rn.f64 %0, %1, %2;" : "=d"(d) : "d"(a), "d"(b));
    return d;
}
__device__ __forceinline__ float cvt_round_trip(float a) {
    double d;
    float f;
    asm volatile("cvt.f64.f32 %0, %1;" : "=d"(d) : "f"(a));
    asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(f) : "d"(d));
    return f;
}
__device__ __forceinline__ uint32_t xor1(uint32_t a, uint32_t b) {
    uint32_t d;
    asm volatile("xor.b32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint64_t pk(float a, float b) {
    return (uint64_t)__float_as_uint(a) | ((uint64_t)__float_as_uint(b) << 32);
}

enum { K_FFMA, K_FFMA2, K_FFMA_XOR, K_FFMA2_XOR, K_DFMA, K_DADD, K_CVT, K_DF_SCALAR, K_DF_PACKED, K_COUNT };
static const char* kNames[K_COUNT] = {"FFMA (16 chains)", "FFMA2 (8 chains)", "FFMA + XOR", "FFMA2 + XOR",
                                      "DFMA", "DADD", "cvt f32->f64->f32", "df butterflies, scalar",
                                      "df butterflies, packed"};
// lane operations per chain step counted for the rate: the XORs are not counted, each of the
// two conversions of a round trip counts one, a butterfly step counts the scalar double-float
// operations (8 lazy sums of 16 and 7 twiddle products of 32)
static const double kOpsPerIter[K_COUNT] = {16, 16, 16, 16, 16, 16, 32, 8 * 16 + 7 * 32, 8 * 16 + 7 * 32};

template <int K>
__global__ void __launch_bounds__(256) k_probe(int n, float s, float* sink) {
    float f[16];
    uint64_t p[8];
    uint32_t q[8];
    double d[16];
#pragma unroll
    for (int i = 0; i < 16; i++) {
        f[i] = s + i;
        d[i] = 0.5 * s + i;
    }
#pragma unroll
    for (int i = 0; i < 8; i++) {
        p[i] = pk(s + i, s - i);
        q[i] = threadIdx.x + i;
    }
    float acc = 0.0f;
    if constexpr (K == K_FFMA || K == K_FFMA_XOR) {
        for (int it = 0; it < n; it++) {
#pragma unroll
            for (int i = 0; i < 16; i++) f[i] = ffma1(f[i], 0.999f, 0.001f);
            if (K == K_FFMA_XOR) {
#pragma unroll
                for (int i = 0; i < 8; i++) q[i] = xor1(q[i], 0x55u);
            }
        }
    } else if constexpr (K == K_FFMA2 || K == K_FFMA2_XOR) {
        const uint64_t c1 = pk(0.999f, 0.998f), c2 = pk(0.001f, 0.002f);
        for (int it = 0; it < n; it++) {
#pragma unroll
            for (int i = 0; i < 8; i++) p[i] = ffma2(p[i], c1, c2);
            if (K == K_FFMA2_XOR) {
#pragma unroll
                for (int i = 0; i < 8; i++) q[i] = xor1(q[i], 0x55u);
            }
        }
    } else if constexpr (K == K_DFMA || K == K_DADD) {
        for (int it = 0; it < n / 16; it++) {
#pragma unroll
            for (int i = 0; i < 16; i++) d[i] = K == K_DFMA ? dfma1(d[i], 0.999, 0.001) : dadd1(d[i], 0.001);
        }
    } else if constexpr (K == K_CVT) {
        for (int it = 0; it < n / 16; it++) {
#pragma unroll
            for (int i = 0; i < 16; i++) f[i] = cvt_round_trip(f[i] + 1.0f);
        }
    } else {
        // one radix-2 layer of lazy sums over 8 values and seven twiddle products per step
        cx<df> v[8];
#pragma unroll
        for (int i = 0; i < 8; i++) v[i] = cmake<df>(df_make(f[i], 1e-9f * f[i]), df_make(f[i + 8], -1e-9f * f[i]));
        const float4 w = make_float4(0.92387953f, -0.38268343f, 1.6e-9f, -2.1e-9f);
        for (int it = 0; it < n / 64; it++) {
#pragma unroll
            for (int i = 0; i < 4; i++) {
                if constexpr (K == K_DF_SCALAR) {
                    const cx<df> a = cmake<df>(df_add_lazy(v[i].re, v[i + 4].re), df_add_lazy(v[i].im, v[i + 4].im));
                    const cx<df> b = cmake<df>(df_sub_lazy(v[i].re, v[i + 4].re), df_sub_lazy(v[i].im, v[i + 4].im));
                    v[i] = a;
                    v[i + 4] = b;
                } else {
                    const cx<df> a = PrecDF::cadd(v[i], v[i + 4]), b = PrecDF::csub(v[i], v[i + 4]);
                    v[i] = a;
                    v[i + 4] = b;
                }
            }
#pragma unroll
            for (int i = 1; i < 8; i++) {
                if constexpr (K == K_DF_SCALAR) {
                    const df wr = df_make(w.x, w.z), wi = df_make(w.y, w.w);
                    v[i] = cmake<df>(df_dot2_lazy(v[i].re, wr, -v[i].im, wi), df_dot2_lazy(v[i].re, wi, v[i].im, wr));
                } else {
                    v[i] = PrecDF::ctw(v[i], w);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 8; i++) acc += v[i].re.hi + v[i].re.lo + v[i].im.hi + v[i].im.lo;
    }
    if constexpr (K == K_DFMA || K == K_DADD) {
#pragma unroll
        for (int i = 0; i < 16; i++) acc += (float)d[i];
    } else if constexpr (K == K_FFMA2 || K == K_FFMA2_XOR) {
#pragma unroll
        for (int i = 0; i < 8; i++) acc += __uint_as_float((uint32_t)p[i]) + __uint_as_float((uint32_t)(p[i] >> 32));
    } else if constexpr (K != K_DF_SCALAR && K != K_DF_PACKED) {
#pragma unroll
        for (int i = 0; i < 16; i++) acc += f[i];
    }
    if constexpr (K == K_FFMA_XOR || K == K_FFMA2_XOR) {
#pragma unroll
        for (int i = 0; i < 8; i++) acc += (float)q[i];
    }
    if (acc == 12345.0f) sink[0] = acc;   // keeps the chains alive; never true for these inputs
}

template <int K>
static float run(int grid, int n, float* sink) {
    k_probe<K><<<grid, 256>>>(n / 8, 1.0f, sink);   // warm-up
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0));
    for (int r = 0; r < 3; r++) k_probe<K><<<grid, 256>>>(n, 1.0f, sink);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    float ms;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    CK(cudaEventDestroy(e0));
    CK(cudaEventDestroy(e1));
    return ms / 3.0f;
}

int main() {
    float* sink;
    CK(cudaMalloc(&sink, sizeof(float)));
    int dev = 0, sms = 0, clk_khz = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev));
    const int grid = sms * 8, n = 8192;
    const double threads = (double)grid * 256;
    printf("%d SMs, %d CTAs x 256 threads, %d chain steps per thread; per SM per clock at the %.0f MHz maximum\n", sms, grid,
           n, clk_khz / 1e3);
    float ms[K_COUNT];
    ms[K_FFMA] = run<K_FFMA>(grid, n, sink);
    ms[K_FFMA2] = run<K_FFMA2>(grid, n, sink);
    ms[K_FFMA_XOR] = run<K_FFMA_XOR>(grid, n, sink);
    ms[K_FFMA2_XOR] = run<K_FFMA2_XOR>(grid, n, sink);
    ms[K_DFMA] = run<K_DFMA>(grid, n, sink);
    ms[K_DADD] = run<K_DADD>(grid, n, sink);
    ms[K_CVT] = run<K_CVT>(grid, n, sink);
    ms[K_DF_SCALAR] = run<K_DF_SCALAR>(grid, n, sink);
    ms[K_DF_PACKED] = run<K_DF_PACKED>(grid, n, sink);
    for (int k = 0; k < K_COUNT; k++) {
        // chain steps: n for the FP32 kernels, n/16 x 16 for FP64 and the conversions, n/64 for the butterflies
        const double iters = (k == K_DF_SCALAR || k == K_DF_PACKED) ? n / 64 : (k >= K_DFMA ? n / 16 : n);
        const double ops = threads * iters * kOpsPerIter[k];
        const double rate = ops / (ms[k] * 1e-3);
        printf("%-26s %9.3f ms %10.1f G lane-op/s %7.1f per SM per clock\n", kNames[k], ms[k], rate * 1e-9,
               rate / sms / (clk_khz * 1e3));
    }
    CK(cudaFree(sink));
    return 0;
}
