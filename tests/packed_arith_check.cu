// packed_arith_check.cu -- the packed FP32x2 double-float arithmetic of kg_arith.cuh (PrecDF)
// against the scalar double-float forms it replaces, on 2^20 seeded complex pairs per case
// with magnitudes spread over 2^-40 .. 2^40, mixed signs, zeros and unnormalised low words.
// Compiled and run by tests/test_gpu_packed.py; prints one line per case:
//   <case> <values compared> <bitwise mismatches> <largest relative difference of hi + lo>
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include "kg_arith.cuh"

using namespace kg;

#define CK(x)                                                                                   \
    do {                                                                                        \
        cudaError_t e_ = (x);                                                                   \
        if (e_ != cudaSuccess) {                                                                \
            printf("CUDA error %s at line %d\n", cudaGetErrorString(e_), __LINE__);             \
            exit(1);                                                                            \
        }                                                                                       \
    } while (0)

enum { C_ADD, C_SUB, C_NORM, C_ROT_P, C_ROT_M, C_ADD_I, C_NEGI_SCALE, C_CUBE, C_SCALE, C_TW, C_COUNT };
static const char* kCase[C_COUNT] = {"cadd", "csub", "cnorm", "crot_plus", "crot_minus", "cadd_i",
                                     "cmul_negi_scale", "ccube", "cscale2", "ctw"};

__device__ __forceinline__ uint32_t mix(uint32_t h) {
    h ^= h >> 16;
    h *= 0x7feb352du;
    h ^= h >> 15;
    h *= 0x846ca68bu;
    h ^= h >> 16;
    return h;
}
// a float with a random sign, significand and exponent in [2^-40, 2^40] (or zero, 1 in 64)
__device__ float rnd_float(uint32_t key) {
    const uint32_t h = mix(key), g = mix(key ^ 0x9e3779b9u);
    if ((g & 63u) == 0u) return 0.0f;
    const int e = (int)(g >> 8) % 81 - 40;
    const float m = 1.0f + (float)(h & 0x7fffffu) * (1.0f / 8388608.0f);
    const float v = ldexpf(m, e);
    return (h & 0x80000000u) ? -v : v;
}
// a double-float with a low word up to 4 ulps of the high one (unnormalised, as the lazy forms leave them)
__device__ df rnd_df(uint32_t key) {
    const float hi = rnd_float(key);
    const uint32_t g = mix(key * 3u + 1u);
    const float ulp = hi == 0.0f ? 0.0f : ldexpf(1.0f, ilogbf(hi) - 23);
    const float lo = ulp * ((float)(g & 0xffffu) / 16384.0f - 2.0f);
    return df_make(hi, lo);
}
__device__ cx<df> rnd_cx(uint32_t key) { return cmake<df>(rnd_df(key * 2u), rnd_df(key * 2u + 1u)); }

__device__ __forceinline__ bool same(df a, df b) {
    return __float_as_uint(a.hi) == __float_as_uint(b.hi) && __float_as_uint(a.lo) == __float_as_uint(b.lo);
}
__device__ __forceinline__ double val(df a) { return (double)a.hi + (double)a.lo; }

__global__ void k_check(int which, int n, unsigned long long* mism, double* maxrel) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t key = (uint32_t)i * 4u + (uint32_t)which * 0x10000000u;
    const cx<df> a = rnd_cx(key), b = rnd_cx(key + 1u);
    const int sg = (i & 1) ? 1 : -1;
    cx<df> p, s;   // packed and scalar results
    switch (which) {
        case C_ADD:
            p = PrecDF::cadd(a, b);
            s = cmake<df>(df_add_lazy(a.re, b.re), df_add_lazy(a.im, b.im));
            break;
        case C_SUB:
            p = PrecDF::csub(a, b);
            s = cmake<df>(df_sub_lazy(a.re, b.re), df_sub_lazy(a.im, b.im));
            break;
        case C_NORM:
            p = PrecDF::cnorm(a);
            s = cmake<df>(df_norm(a.re), df_norm(a.im));
            break;
        case C_ROT_P:
        case C_ROT_M: {
            // x (1 + sg i)/sqrt2 = (x.re - sg x.im, x.im + sg x.re)/sqrt2 and
            // x (-1 + sg i)/sqrt2 = (-sg x.im - x.re, sg x.re - x.im)/sqrt2
            const df r = PrecDF::rsqrt2();
            const df ni = df_make(-sg * a.im.hi, -sg * a.im.lo), nr = df_make(sg * a.re.hi, sg * a.re.lo);
            if (which == C_ROT_P) {
                p = PrecDF::crot(a, sg, false);
                s = cmake<df>(df_mul_lazy(df_add_lazy(a.re, ni), r), df_mul_lazy(df_add_lazy(a.im, nr), r));
            } else {
                p = PrecDF::crot(a, sg, true);
                s = cmake<df>(df_mul_lazy(df_sub_lazy(ni, a.re), r), df_mul_lazy(df_sub_lazy(nr, a.im), r));
            }
            break;
        }
        case C_ADD_I:   // a + i b
            p = PrecDF::cadd_i(a, b);
            s = cmake<df>(df_sub_lazy(a.re, b.im), df_add_lazy(a.im, b.re));
            break;
        case C_NEGI_SCALE:   // (-i a) / 2
            p = PrecDF::cscale2(PrecDF::cmul_negi(a), 0.5);
            s = cmake<df>(df_scale2(a.im, 0.5f), df_scale2(-a.re, 0.5f));
            break;
        case C_CUBE: {   // operands scaled by 2^-20 so that lam x^3 stays below the float range
            const df lam = rnd_df(key + 7u);
            const cx<df> x = cmake<df>(df_scale2(a.re, 0x1p-20f), df_scale2(a.im, 0x1p-20f));
            p = PrecDF::ccube(x, lam);
            s = cmake<df>(PrecDF::cube(x.re, lam), PrecDF::cube(x.im, lam));
            break;
        }
        case C_SCALE:
            p = PrecDF::cscale2(a, 0x1p-27);
            s = cmake<df>(df_scale2(a.re, 0x1p-27f), df_scale2(a.im, 0x1p-27f));
            break;
        default: {   // twiddle product with a unit-modulus w; the imaginary lane adds its
                     // low-order terms in another order, so it is compared by value
            const float ang = (float)(mix(key + 5u) & 0xffffu) * (6.2831853f / 65536.0f);
            const double c = cos((double)ang), sn = sin((double)ang);
            const float ch = (float)c, sh = (float)sn;
            const float4 wraw = make_float4(ch, sh, (float)(c - (double)ch), (float)(sn - (double)sh));
            const PrecDF::S ws = wraw;   // (re.hi, im.hi, re.lo, im.lo)
            const cx<df> w = PrecDF::load(ws);
            p = PrecDF::ctw(a, PrecDF::twl(ws, -1));
            s = cmake<df>(df_dot2_lazy(a.re, w.re, -a.im, w.im), df_dot2_lazy(a.re, w.im, a.im, w.re));
            break;
        }
    }
    const bool bit = which == C_TW ? same(p.re, s.re) : (same(p.re, s.re) && same(p.im, s.im));
    if (!bit) atomicAdd(mism, 1ull);
    // value difference relative to the size of the operands
    const double scale = fabs(val(a.re)) + fabs(val(a.im)) + fabs(val(b.re)) + fabs(val(b.im)) + 1e-300;
    const double d = fmax(fabs(val(p.re) - val(s.re)), fabs(val(p.im) - val(s.im))) / scale;
    if (d > 0.0) {
        // atomic max on the bit pattern of a non-negative double
        atomicMax(reinterpret_cast<unsigned long long*>(maxrel), (unsigned long long)__double_as_longlong(d));
    }
}

int main() {
    const int n = 1 << 20;
    unsigned long long* mism;
    double* maxrel;
    CK(cudaMalloc(&mism, sizeof(unsigned long long) * C_COUNT));
    CK(cudaMalloc(&maxrel, sizeof(double) * C_COUNT));
    CK(cudaMemset(mism, 0, sizeof(unsigned long long) * C_COUNT));
    CK(cudaMemset(maxrel, 0, sizeof(double) * C_COUNT));
    for (int c = 0; c < C_COUNT; c++) k_check<<<(n + 255) / 256, 256>>>(c, n, mism + c, maxrel + c);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    unsigned long long hm[C_COUNT];
    double hr[C_COUNT];
    CK(cudaMemcpy(hm, mism, sizeof(hm), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hr, maxrel, sizeof(hr), cudaMemcpyDeviceToHost));
    for (int c = 0; c < C_COUNT; c++) printf("%s %d %llu %.3e\n", kCase[c], n, hm[c], hr[c]);
    CK(cudaFree(mism));
    CK(cudaFree(maxrel));
    return 0;
}
