// kg_mlp.cu -- the blow-up ranker network: training and inference on the GPU.
//
// The paper motivates parametric studies of blow-up (section 1) but has no learned
// component; this network is the project's.  Network 6 -> 128 -> 128 -> 2 (ReLU),
// heads z0 = blow-up logit and z1 = predicted log blow-up time.  Loss, mean over the
// batch: BCE(z0, y) + y (z1 - l)^2 + (1 - y) relu(log T - z1)^2 (runs that did not
// blow up by T only bound t_b from below).  Adam on FP32 master weights.
//
// Arithmetic: BF16 operands (inputs, weights, activations h1, h2 and the activation
// gradients dz, dh2, dh1, rounded to nearest even where they are stored) on the
// tensor cores with FP32 accumulation (mma.sync m16n8k16); biases, the loss and the
// weight gradients are FP32.  One CTA of 8 warps handles a tile of 128 batch rows
// with all weights in shared memory; warp w owns rows 16w .. 16w+15.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/kg.h"
#include "kg_launch.h"

namespace {

constexpr int DIN = 6, DH = 128, DOUT = 2;
constexpr int KIN = 16;                          // padded input width (one MMA k-step)
constexpr int K3 = 16;                           // padded output width of W3 / dz
constexpr int BT = 128;                          // batch rows per CTA
constexpr int NTH = 256;
constexpr int NPARAM = DIN * DH + DH + DH * DH + DH + DH * DOUT + DOUT;
// offsets of the tensors in the flat parameter vector (order W1, b1, W2, b2, W3, b3)
constexpr int OW1 = 0, OB1 = OW1 + DIN * DH, OW2 = OB1 + DH, OB2 = OW2 + DH * DH, OW3 = OB2 + DH,
              OB3 = OW3 + DH * DOUT;

typedef unsigned short bf;   // raw bfloat16 bits

__device__ __forceinline__ bf to_bf(float f) { return __bfloat16_as_ushort(__float2bfloat16_rn(f)); }
__device__ __forceinline__ float from_bf(bf b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

// C(16x8, fp32) += A(16x16) B(16x8); element (r, c) of A at A[r*ars + c*acs], element
// (k, n) of B at B[k*brs + n*bcs]; fragment layout of mma.m16n8k16 (g = lane/4, t = lane%4):
// A regs {(g, 2t..2t+1), (g+8, 2t..), (g, 2t+8..), (g+8, 2t+8..)}, B regs {(2t..2t+1, g), (2t+8.., g)},
// C {(g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1)}.
__device__ __forceinline__ void mma_16x8x16(float c[4], const bf* A, int ars, int acs, int m0, int k0, const bf* B,
                                            int brs, int bcs, int n0) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    unsigned a[4], b[2];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int row = m0 + g + (r & 1) * 8, col = k0 + 2 * t + (r >> 1) * 8;
        const unsigned lo = A[row * ars + col * acs], hi = A[row * ars + (col + 1) * acs];
        a[r] = lo | (hi << 16);
    }
#pragma unroll
    for (int r = 0; r < 2; r++) {
        const int k = k0 + 2 * t + r * 8, n = n0 + g;
        const unsigned lo = B[k * brs + n * bcs], hi = B[(k + 1) * brs + n * bcs];
        b[r] = lo | (hi << 16);
    }
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct Smem {
    bf x[BT * KIN];
    bf w1[KIN * DH];
    bf w2[DH * DH];
    bf w3[DH * K3];
    bf h1[BT * DH];
    bf h2[BT * DH];     // reused for dh1 in the backward pass
    bf dz[BT * K3];
    bf dh2[BT * DH];
    float b1[DH], b2[DH], b3[DOUT];
};

struct Params {   // device pointers
    const float* master;     // NPARAM fp32
    const bf* w1b;           // KIN x DH
    const bf* w2b;           // DH x DH
    const bf* w3b;           // DH x K3
};

// load the weights and the input tile; rows beyond n (or gathered through idx) are zero
__device__ void load_tile(Smem& s, const Params& P, const float* X, const int* idx, int n, int row0) {
    for (int i = threadIdx.x; i < KIN * DH; i += NTH) s.w1[i] = P.w1b[i];
    for (int i = threadIdx.x; i < DH * DH; i += NTH) s.w2[i] = P.w2b[i];
    for (int i = threadIdx.x; i < DH * K3; i += NTH) s.w3[i] = P.w3b[i];
    for (int i = threadIdx.x; i < DH; i += NTH) {
        s.b1[i] = P.master[OB1 + i];
        s.b2[i] = P.master[OB2 + i];
    }
    if (threadIdx.x < DOUT) s.b3[threadIdx.x] = P.master[OB3 + threadIdx.x];
    for (int i = threadIdx.x; i < BT * KIN; i += NTH) {
        const int r = i / KIN, c = i % KIN, row = row0 + r;
        float v = 0.f;
        if (c < DIN && row < n) v = X[(size_t)(idx ? idx[row] : row) * DIN + c];
        s.x[i] = to_bf(v);
    }
    for (int i = threadIdx.x; i < BT * K3; i += NTH) s.dz[i] = 0;
    __syncthreads();
}

// forward for the warp's 16 rows; returns z in c3 (fragment of the 16x8 output tile)
__device__ void forward_rows(Smem& s, float c3[4]) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int r0 = 16 * w;
    for (int nt = 0; nt < DH / 8; nt++) {   // h1 = relu(x W1 + b1)
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma_16x8x16(c, s.x, KIN, 1, r0, 0, s.w1, DH, 1, 8 * nt);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int row = r0 + g + (q >> 1) * 8, col = 8 * nt + 2 * t + (q & 1);
            s.h1[row * DH + col] = to_bf(fmaxf(c[q] + s.b1[col], 0.f));
        }
    }
    __syncwarp();
    for (int nt = 0; nt < DH / 8; nt++) {   // h2 = relu(h1 W2 + b2)
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        for (int kt = 0; kt < DH / 16; kt++) mma_16x8x16(c, s.h1, DH, 1, r0, 16 * kt, s.w2, DH, 1, 8 * nt);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int row = r0 + g + (q >> 1) * 8, col = 8 * nt + 2 * t + (q & 1);
            s.h2[row * DH + col] = to_bf(fmaxf(c[q] + s.b2[col], 0.f));
        }
    }
    __syncwarp();
    for (int q = 0; q < 4; q++) c3[q] = 0.f;   // z = h2 W3 + b3 (columns 0, 1 of the tile)
    for (int kt = 0; kt < DH / 16; kt++) mma_16x8x16(c3, s.h2, DH, 1, r0, 16 * kt, s.w3, K3, 1, 0);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int col = 2 * t + (q & 1);
        if (col < DOUT) c3[q] += s.b3[col];
    }
}

__global__ void __launch_bounds__(NTH) k_mlp_forward(Params P, const float* X, int n, float* z) {
    extern __shared__ __align__(16) unsigned char raw[];
    Smem& s = *reinterpret_cast<Smem*>(raw);
    const int row0 = blockIdx.x * BT;
    load_tile(s, P, X, nullptr, n, row0);
    float c3[4];
    forward_rows(s, c3);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    if (t == 0) {   // columns 0 and 1 live in c3[0], c3[1] (row g) and c3[2], c3[3] (row g+8)
        const int ra = row0 + 16 * w + g, rb = ra + 8;
        if (ra < n) { z[2 * (size_t)ra] = c3[0]; z[2 * (size_t)ra + 1] = c3[1]; }
        if (rb < n) { z[2 * (size_t)rb] = c3[2]; z[2 * (size_t)rb + 1] = c3[3]; }
    }
}

// gradients of the mean loss over rows idx[0..n) (idx may be NULL: rows 0..n), scaled
// by 1/n_total, accumulated into grad (fp32, atomics); the loss sum into *loss
__global__ void __launch_bounds__(NTH) k_mlp_backward(Params P, const float* X, const float* Y, const float* ELL,
                                                      const int* idx, int n, float inv_n, float logT, float* grad,
                                                      float* loss) {
    extern __shared__ __align__(16) unsigned char raw[];
    Smem& s = *reinterpret_cast<Smem*>(raw);
    const int row0 = blockIdx.x * BT;
    load_tile(s, P, X, idx, n, row0);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int r0 = 16 * w;
    float c3[4];
    forward_rows(s, c3);

    // dz = dL/dz per row (threads with t == 0 hold both heads of rows g and g+8)
    float lsum = 0.f;
    float db3a = 0.f, db3b = 0.f;
    if (t == 0) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int r = r0 + g + 8 * h, row = row0 + r;
            float d0 = 0.f, d1 = 0.f;
            if (row < n) {
                const int src = idx ? idx[row] : row;
                const float y = Y[src], ell = ELL[src];
                const float z0 = c3[2 * h], z1 = c3[2 * h + 1];
                const float sig = 1.f / (1.f + expf(-z0));
                const float cens = fmaxf(logT - z1, 0.f);
                lsum += fmaxf(z0, 0.f) - y * z0 + log1pf(expf(-fabsf(z0))) + y * (z1 - ell) * (z1 - ell) +
                        (1.f - y) * cens * cens;
                d0 = (sig - y) * inv_n;
                d1 = (2.f * y * (z1 - ell) - 2.f * (1.f - y) * cens) * inv_n;
            }
            const bf b0 = to_bf(d0), b1 = to_bf(d1);
            s.dz[r * K3 + 0] = b0;
            s.dz[r * K3 + 1] = b1;
            db3a += from_bf(b0);
            db3b += from_bf(b1);
        }
    }
    // loss and db3: warp sums, one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        db3a += __shfl_xor_sync(0xffffffffu, db3a, o);
        db3b += __shfl_xor_sync(0xffffffffu, db3b, o);
    }
    if (lane == 0) {
        atomicAdd(loss, lsum);
        atomicAdd(grad + OB3, db3a);
        atomicAdd(grad + OB3 + 1, db3b);
    }
    __syncthreads();

    // dW3 = h2^T dz: warp w owns features 16w..16w+15, k runs over the tile's 128 rows
    {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        for (int kt = 0; kt < BT / 16; kt++) mma_16x8x16(c, s.h2, 1, DH, 16 * w, 16 * kt, s.dz, K3, 1, 0);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int f = 16 * w + g + (q >> 1) * 8, col = 2 * t + (q & 1);
            if (col < DOUT) atomicAdd(grad + OW3 + f * DOUT + col, c[q]);
        }
    }
    // dh2 = (dz W3^T) masked by h2 > 0, for the warp's rows
    for (int nt = 0; nt < DH / 8; nt++) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma_16x8x16(c, s.dz, K3, 1, r0, 0, s.w3, 1, K3, 8 * nt);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int row = r0 + g + (q >> 1) * 8, col = 8 * nt + 2 * t + (q & 1);
            s.dh2[row * DH + col] = from_bf(s.h2[row * DH + col]) > 0.f ? to_bf(c[q]) : (bf)0;
        }
    }
    __syncthreads();   // every row of dh2 is needed below; h2 is free from here on
    // dh1 = (dh2 W2^T) masked by h1 > 0, written over h2
    bf* dh1 = s.h2;
    for (int nt = 0; nt < DH / 8; nt++) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        for (int kt = 0; kt < DH / 16; kt++) mma_16x8x16(c, s.dh2, DH, 1, r0, 16 * kt, s.w2, 1, DH, 8 * nt);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int row = r0 + g + (q >> 1) * 8, col = 8 * nt + 2 * t + (q & 1);
            dh1[row * DH + col] = from_bf(s.h1[row * DH + col]) > 0.f ? to_bf(c[q]) : (bf)0;
        }
    }
    // dW2 = h1^T dh2: warp w owns rows 16w.. of dW2, all 128 columns
    for (int nt = 0; nt < DH / 8; nt++) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        for (int kt = 0; kt < BT / 16; kt++) mma_16x8x16(c, s.h1, 1, DH, 16 * w, 16 * kt, s.dh2, DH, 1, 8 * nt);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int f1 = 16 * w + g + (q >> 1) * 8, f2 = 8 * nt + 2 * t + (q & 1);
            atomicAdd(grad + OW2 + f1 * DH + f2, c[q]);
        }
    }
    __syncthreads();   // dh1 complete
    // dW1 = x^T dh1: one 16-row tile (inputs), warp w owns columns 16w .. 16w+15
    for (int h = 0; h < 2; h++) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        const int n0 = 16 * w + 8 * h;
        for (int kt = 0; kt < BT / 16; kt++) mma_16x8x16(c, s.x, 1, KIN, 0, 16 * kt, dh1, DH, 1, n0);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int i = g + (q >> 1) * 8, f = n0 + 2 * t + (q & 1);
            if (i < DIN) atomicAdd(grad + OW1 + i * DH + f, c[q]);
        }
    }
    // db2, db1: column sums over the tile
    if (threadIdx.x < DH) {
        float a = 0.f, b = 0.f;
        for (int r = 0; r < BT; r++) {
            a += from_bf(s.dh2[r * DH + threadIdx.x]);
            b += from_bf(dh1[r * DH + threadIdx.x]);
        }
        atomicAdd(grad + OB2 + threadIdx.x, a);
        atomicAdd(grad + OB1 + threadIdx.x, b);
    }
}

// Adam on the master weights, then refresh the bf16 copies (padded shapes) and clear grad
__global__ void k_mlp_adam(float* master, float* grad, float* m, float* v, float lr, float b1, float b2, float eps,
                           float c1, float c2, bf* w1b, bf* w2b, bf* w3b, int apply) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x) {
        float wv = master[i];
        if (apply) {
            const float gv = grad[i];
            const float mv = b1 * m[i] + (1.f - b1) * gv;
            const float vv = b2 * v[i] + (1.f - b2) * gv * gv;
            m[i] = mv;
            v[i] = vv;
            wv -= lr * (mv * c1) / (sqrtf(vv * c2) + eps);
            master[i] = wv;
            grad[i] = 0.f;
        }
        if (i < OB1) {
            const int r = i / DH, c = i % DH;
            w1b[r * DH + c] = to_bf(wv);
        } else if (i >= OW2 && i < OB2) {
            w2b[i - OW2] = to_bf(wv);
        } else if (i >= OW3 && i < OB3) {
            const int r = (i - OW3) / DOUT, c = (i - OW3) % DOUT;
            w3b[r * K3 + c] = to_bf(wv);
        }
    }
}

struct Mlp {
    float* master = nullptr;
    float* grad = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    bf* w1b = nullptr;
    bf* w2b = nullptr;
    bf* w3b = nullptr;
    float* loss = nullptr;
    long long t = 0;
    std::vector<void*> allocs;
};
Mlp* g_mlp = nullptr;

int mfail(int code, const std::string& msg) { return kg::set_last_error(code, msg); }

#define KG_MCK(call)                                                                               \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return mfail(KG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int mlp_alloc(Mlp* M, void** p, size_t b) {
    if (cudaMalloc(p, b) != cudaSuccess) {
        cudaGetLastError();
        return mfail(KG_ENOMEM, "mlp allocation");
    }
    cudaMemset(*p, 0, b);
    M->allocs.push_back(*p);
    return KG_OK;
}

void mlp_destroy(Mlp* M) {
    if (!M) return;
    cudaDeviceSynchronize();
    for (void* p : M->allocs) cudaFree(p);
    delete M;
}

int mlp_ensure() {
    if (g_mlp) return KG_OK;
    Mlp* M = new Mlp();
    int rc = mlp_alloc(M, (void**)&M->master, sizeof(float) * NPARAM);
    if (!rc) rc = mlp_alloc(M, (void**)&M->grad, sizeof(float) * NPARAM);
    if (!rc) rc = mlp_alloc(M, (void**)&M->m, sizeof(float) * NPARAM);
    if (!rc) rc = mlp_alloc(M, (void**)&M->v, sizeof(float) * NPARAM);
    if (!rc) rc = mlp_alloc(M, (void**)&M->w1b, sizeof(bf) * KIN * DH);
    if (!rc) rc = mlp_alloc(M, (void**)&M->w2b, sizeof(bf) * DH * DH);
    if (!rc) rc = mlp_alloc(M, (void**)&M->w3b, sizeof(bf) * DH * K3);
    if (!rc) rc = mlp_alloc(M, (void**)&M->loss, sizeof(float));
    if (rc) {
        mlp_destroy(M);
        return rc;
    }
    g_mlp = M;
    return KG_OK;
}

Params params_of(const Mlp* M) { return Params{M->master, M->w1b, M->w2b, M->w3b}; }

int refresh_bf16(Mlp* M) {
    k_mlp_adam<<<72, 256>>>(M->master, M->grad, M->m, M->v, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, M->w1b, M->w2b, M->w3b, 0);
    KG_MCK(cudaGetLastError());
    return KG_OK;
}

int set_smem_once() {
    static bool done = false;
    if (done) return KG_OK;
    KG_MCK(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem)));
    KG_MCK(cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem)));
    done = true;
    return KG_OK;
}

// device copies of host training data
struct DevData {
    float *X = nullptr, *Y = nullptr, *E = nullptr;
    int* idx = nullptr;
    ~DevData() {
        cudaFree(X);
        cudaFree(Y);
        cudaFree(E);
        cudaFree(idx);
    }
};

int upload(DevData& d, const float* X, const float* y, const float* ell, int n) {
    if (cudaMalloc((void**)&d.X, sizeof(float) * DIN * (size_t)n) != cudaSuccess ||
        (y && cudaMalloc((void**)&d.Y, sizeof(float) * (size_t)n) != cudaSuccess) ||
        (ell && cudaMalloc((void**)&d.E, sizeof(float) * (size_t)n) != cudaSuccess) ||
        cudaMalloc((void**)&d.idx, sizeof(int) * (size_t)n) != cudaSuccess) {
        cudaGetLastError();
        return mfail(KG_ENOMEM, "mlp data allocation");
    }
    KG_MCK(cudaMemcpy(d.X, X, sizeof(float) * DIN * (size_t)n, cudaMemcpyHostToDevice));
    if (y) KG_MCK(cudaMemcpy(d.Y, y, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice));
    if (ell) KG_MCK(cudaMemcpy(d.E, ell, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice));
    return KG_OK;
}

}  // namespace

extern "C" {

int kg_mlp_set_params(const float* params) {
    if (!params) return mfail(KG_EINVAL, "NULL params");
    for (int i = 0; i < NPARAM; i++)
        if (!std::isfinite(params[i])) return mfail(KG_EINVAL, "non-finite parameter");
    int rc = mlp_ensure();
    if (rc) return rc;
    KG_MCK(cudaMemcpy(g_mlp->master, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
    KG_MCK(cudaMemset(g_mlp->grad, 0, sizeof(float) * NPARAM));
    KG_MCK(cudaMemset(g_mlp->m, 0, sizeof(float) * NPARAM));
    KG_MCK(cudaMemset(g_mlp->v, 0, sizeof(float) * NPARAM));
    g_mlp->t = 0;
    return refresh_bf16(g_mlp);
}

int kg_mlp_get_params(float* params) {
    if (!g_mlp) return mfail(KG_ESTATE, "kg_mlp_get_params before kg_mlp_set_params");
    if (!params) return mfail(KG_EINVAL, "NULL params");
    KG_MCK(cudaMemcpy(params, g_mlp->master, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
    return KG_OK;
}

int kg_mlp_predict(const float* X, int n, float* p_blowup, float* logt) {
    if (!g_mlp) return mfail(KG_ESTATE, "kg_mlp_predict before kg_mlp_set_params");
    if (!X || n < 1) return mfail(KG_EINVAL, "bad arguments");
    int rc = set_smem_once();
    if (rc) return rc;
    DevData d;
    rc = upload(d, X, nullptr, nullptr, n);
    if (rc) return rc;
    float* z = nullptr;
    if (cudaMalloc((void**)&z, sizeof(float) * 2 * (size_t)n) != cudaSuccess) return mfail(KG_ENOMEM, "mlp output");
    k_mlp_forward<<<(n + BT - 1) / BT, NTH, sizeof(Smem)>>>(params_of(g_mlp), d.X, n, z);
    cudaError_t e = cudaGetLastError();
    std::vector<float> h(2 * (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), z, sizeof(float) * 2 * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(z);
    if (e != cudaSuccess) return mfail(KG_ECUDA, std::string("mlp forward: ") + cudaGetErrorString(e));
    for (int i = 0; i < n; i++) {
        if (p_blowup) p_blowup[i] = 1.f / (1.f + std::exp(-h[2 * (size_t)i]));
        if (logt) logt[i] = h[2 * (size_t)i + 1];
    }
    return KG_OK;
}

int kg_mlp_grad(const float* X, const float* y, const float* logt, int n, double T, float* grad, double* loss) {
    if (!g_mlp) return mfail(KG_ESTATE, "kg_mlp_grad before kg_mlp_set_params");
    if (!X || !y || !logt || n < 1 || !(T > 0.0)) return mfail(KG_EINVAL, "bad arguments");
    int rc = set_smem_once();
    if (rc) return rc;
    DevData d;
    rc = upload(d, X, y, logt, n);
    if (rc) return rc;
    KG_MCK(cudaMemset(g_mlp->grad, 0, sizeof(float) * NPARAM));
    KG_MCK(cudaMemset(g_mlp->loss, 0, sizeof(float)));
    k_mlp_backward<<<(n + BT - 1) / BT, NTH, sizeof(Smem)>>>(params_of(g_mlp), d.X, d.Y, d.E, nullptr, n,
                                                             1.f / (float)n, (float)std::log(T), g_mlp->grad,
                                                             g_mlp->loss);
    KG_MCK(cudaGetLastError());
    if (grad) KG_MCK(cudaMemcpy(grad, g_mlp->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
    float l = 0.f;
    KG_MCK(cudaMemcpy(&l, g_mlp->loss, sizeof(float), cudaMemcpyDeviceToHost));
    if (loss) *loss = (double)l / n;
    KG_MCK(cudaMemset(g_mlp->grad, 0, sizeof(float) * NPARAM));
    return KG_OK;
}

int kg_mlp_train(const float* X, const float* y, const float* logt, int n, const kg_mlp_cfg* cfg, double* final_loss) {
    if (!g_mlp) return mfail(KG_ESTATE, "kg_mlp_train before kg_mlp_set_params");
    if (!X || !y || !logt || n < 1 || !cfg || cfg->epochs < 0 || cfg->batch < 1 || !(cfg->lr > 0.0) ||
        !(cfg->T > 0.0))
        return mfail(KG_EINVAL, "bad arguments");
    int rc = set_smem_once();
    if (rc) return rc;
    DevData d;
    rc = upload(d, X, y, logt, n);
    if (rc) return rc;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const int batch = cfg->batch < n ? cfg->batch : n;
    std::vector<int> perm(n);
    unsigned long long st = cfg->seed ? cfg->seed : 0x9E3779B97F4A7C15ull;
    float lastloss = 0.f;
    for (int ep = 0; ep < cfg->epochs; ep++) {
        for (int i = 0; i < n; i++) perm[i] = i;
        for (int i = n - 1; i > 0; i--) {   // Fisher-Yates with a xorshift64 stream
            st ^= st << 13;
            st ^= st >> 7;
            st ^= st << 17;
            const int j = (int)(st % (unsigned long long)(i + 1));
            const int tmp = perm[i];
            perm[i] = perm[j];
            perm[j] = tmp;
        }
        KG_MCK(cudaMemcpy(d.idx, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
        KG_MCK(cudaMemset(g_mlp->loss, 0, sizeof(float)));
        for (int b0 = 0; b0 + batch <= n; b0 += batch) {
            k_mlp_backward<<<(batch + BT - 1) / BT, NTH, sizeof(Smem)>>>(params_of(g_mlp), d.X, d.Y, d.E, d.idx + b0,
                                                                         batch, 1.f / (float)batch,
                                                                         (float)std::log(cfg->T), g_mlp->grad,
                                                                         g_mlp->loss);
            g_mlp->t += 1;
            const float c1 = 1.f / (1.f - std::pow(b1, (float)g_mlp->t));
            const float c2 = 1.f / (1.f - std::pow(b2, (float)g_mlp->t));
            k_mlp_adam<<<72, 256>>>(g_mlp->master, g_mlp->grad, g_mlp->m, g_mlp->v, (float)cfg->lr, b1, b2, eps, c1,
                                    c2, g_mlp->w1b, g_mlp->w2b, g_mlp->w3b, 1);
        }
        KG_MCK(cudaGetLastError());
        KG_MCK(cudaMemcpy(&lastloss, g_mlp->loss, sizeof(float), cudaMemcpyDeviceToHost));
        lastloss /= (float)((n / batch) * batch);
    }
    KG_MCK(cudaDeviceSynchronize());
    if (final_loss) *final_loss = lastloss;
    return KG_OK;
}

int kg_mlp_adam_step(const float* grad, double lr) {
    if (!g_mlp) return mfail(KG_ESTATE, "kg_mlp_adam_step before kg_mlp_set_params");
    if (!grad || !(lr > 0.0)) return mfail(KG_EINVAL, "bad arguments");
    KG_MCK(cudaMemcpy(g_mlp->grad, grad, sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
    g_mlp->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - std::pow(b1, (float)g_mlp->t)), c2 = 1.f / (1.f - std::pow(b2, (float)g_mlp->t));
    k_mlp_adam<<<72, 256>>>(g_mlp->master, g_mlp->grad, g_mlp->m, g_mlp->v, (float)lr, b1, b2, 1e-8f, c1, c2,
                            g_mlp->w1b, g_mlp->w2b, g_mlp->w3b, 1);
    KG_MCK(cudaGetLastError());
    KG_MCK(cudaDeviceSynchronize());
    return KG_OK;
}

int kg_mlp_param_count(void) { return NPARAM; }

int kg_mlp_finalize(void) {
    mlp_destroy(g_mlp);
    g_mlp = nullptr;
    return KG_OK;
}

}  // extern "C"
