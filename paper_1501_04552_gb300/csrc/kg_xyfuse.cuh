// kg_xyfuse.cuh -- inverse y, x and forward y passes of one z-plane fused in a
// thread-block cluster (FP32 work array).
//
// Between two z passes a step runs three in-place passes over W: the inverse y
// transform that ends step n, then the x pass (C2R, cube of section 1.1.2's
// nonlinearity, R2C) and the forward y transform that begin step n+1.  Each of them
// reads and writes all of W once.  All three only mix values within one z-plane
// (N rows y by N/2+1 columns kx; 1.05 MB in FP32 at N = 512), and a plane fits in the
// shared memory of a cluster of CL CTAs on CL SMs (distributed shared memory).  So a
// cluster loads a plane once, runs the three transforms on it, and writes it back once:
// 2 W of HBM traffic instead of 6 W.
//
// CTA r of a cluster holds a slab of the plane: all N rows of the kx columns
// [r CW, (r+1) CW) (the last CTA also holds the Nyquist column kx = N/2), row pitch
// LDC.  The y transforms are column transforms of its own slab (the FFT engine of the
// column passes, exchanging through the slab itself).  For the x transforms CTA r
// takes the rows [r RPC, (r+1) RPC); one x-line is spread over the slabs of all CL
// CTAs, and its threads read and write it through distributed shared memory (the
// x-line body of the x pass, with an element accessor in place of a pointer).  Two
// cluster barriers per plane order the phases: after the inverse y transforms (every
// slab is ready to be read) and after the x transforms (every remote write has landed
// before the slab's owner transforms it again).  Every CTA of a cluster takes the same
// planes, so every CTA reaches every barrier.
//
// Statistics of u^n (max |u|, sum u^4) are those of the x pass, one partial per CTA.
#pragma once
#include <cooperative_groups.h>

#include "kg_kernels.cuh"

namespace kg {

namespace cgx = cooperative_groups;

template <int N, int CL>
struct XyShape {
    static constexpr int NX = N / 2 + 1;
    static constexpr int CW = (N / 2) / CL;          // columns per slab (the last slab: CW + 1)
    static constexpr int LDC = CW + 1;                // slab row pitch, in values
    static constexpr int RPC = N / CL;                // x-lines per CTA
    static constexpr int TY = N / 8;                  // threads per column transform
    static constexpr int TX = N / 16;                 // threads per x-line (N/2-point transform)
    static constexpr int YROUNDS = (LDC * TY + 1023) / 1024;
    static constexpr int YCOLS = (LDC + YROUNDS - 1) / YROUNDS;   // column transforms per round
    static constexpr int NT = (YCOLS * TY + 31) / 32 * 32;        // threads per CTA
    static constexpr int XLINES = NT / TX;                         // x-lines per round
    static constexpr int XROUNDS = (RPC + XLINES - 1) / XLINES;
    static constexpr int PADM = XShape<N>::PADM;                   // x-line exchange slots
    static constexpr int SLAB = N * LDC;                           // values
    static constexpr int XBUF = XLINES * PADM;                     // values
    static constexpr int YIDLE = NT / TY;                          // column slots of a round's threads
    static constexpr int DUMMY = N * YIDLE;                        // values, inside the x buffers
    static_assert(CW >= 1 && (N / 2) % CL == 0 && N % CL == 0, "slabs and x-line blocks tile the plane");
    static_assert(DUMMY <= XBUF, "idle column transforms exchange inside the x-line buffers");
    static_assert(NT <= 1024, "one CTA");
    // resident CTAs per SM compiled for: two when both fit in an SM's shared memory
    static constexpr int MINB = 2 * (SLAB + XBUF) * 8 + 2048 <= 232448 ? 2 : 1;
};

// every thread of every CTA of the cluster: the memory operations before it (stores into
// other CTAs' shared memory included) are visible to every thread after it
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("fence.acq_rel.cluster;\n" ::: "memory");
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// the column view of one column transform: rows of the slab (or of the idle area)
template <class P>
struct SlabCol {
    typename P::S* base;
    int ld;
    __device__ __forceinline__ void put(int row, cx<typename P::R> v) { base[row * ld] = P::pack(v); }
    __device__ __forceinline__ cx<typename P::R> get(int row) const { return P::load(base[row * ld]); }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// one element of an x-line in the cluster's distributed shared memory; an idle line
// (p == nullptr) reads zeros and drops writes
template <class S>
struct DsmemRef {
    S* p;
    __device__ __forceinline__ operator S() const {
        if (p) return *p;
        S z;
        z.x = 0.f;
        z.y = 0.f;
        return z;
    }
    __device__ __forceinline__ DsmemRef& operator=(const S& v) {
        if (p) *p = v;
        return *this;
    }
};

// x-line y of the plane: element kx lives in slab r = min(kx / CW, CL - 1) at column
// kx - r CW of row y
template <class S, int N, int CL>
struct ClusterLine {
    S* slab;   // this CTA's slab (a shared-memory address; mapped to slab r per access)
    int y;
    bool active;
    __device__ __forceinline__ DsmemRef<S> operator[](int kx) const {
        typedef XyShape<N, CL> X;
        if (!active) return DsmemRef<S>{nullptr};
        int r = kx / X::CW;
        r = r < CL - 1 ? r : CL - 1;
        S* local = slab + y * X::LDC + (kx - r * X::CW);
        return DsmemRef<S>{cgx::this_cluster().map_shared_rank(local, (unsigned)r)};
    }
};

// DO_YI: start with the inverse y transforms (W holds the output of a z pass); without
// it W already holds the y-inverse (the first step after set-up or a previous call).
template <int N, int CL, bool DO_YI>
__global__ void __launch_bounds__(XyShape<N, CL>::NT, XyShape<N, CL>::MINB)
    k_xy_cluster(float2* __restrict__ W, KgDev* __restrict__ dev, double* __restrict__ part_sum,
                 double* __restrict__ part_max, const float2* __restrict__ tw, double scale, double lam) {
    typedef PrecF32 P;
    typedef float2 S;
    typedef cx<float> C;
    typedef XyShape<N, CL> X;
    constexpr int NX = X::NX, CW = X::CW, LDC = X::LDC, TY = X::TY, TX = X::TX;
    extern __shared__ __align__(16) unsigned char smraw[];
    S* slab = reinterpret_cast<S*>(smraw);
    S* xbuf = slab + X::SLAB;
    __shared__ double red[96];
    __shared__ unsigned long long kred[X::NT / 32];
    cgx::cluster_group cluster = cgx::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int nclusters = (int)(gridDim.x / CL);
    const int cid = (int)(blockIdx.x / CL);
    const int c0 = rank * CW;
    const int ncols = rank == CL - 1 ? CW + 1 : CW;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NWARPS = X::NT / 32;
    const bool want_sum = kg_recording(dev) || dev->record_p;
    const float rlam = P::from_f64(lam);
    Stats<P> st;
    st.init();

    // column transforms of this slab, sign sg, in rounds of YCOLS columns
    auto y_transforms = [&](int sg) {
#pragma unroll 1
        for (int yr = 0; yr < X::YROUNDS; yr++) {
            const int cl = yr * X::YCOLS + tid / TY, j = tid % TY;
            const bool act = cl < ncols;
            SlabCol<P> col{act ? slab + cl : xbuf + tid / TY, act ? LDC : X::YIDLE};
            C v[8];
#pragma unroll
            for (int s = 0; s < 8; s++) v[s] = col.get(j + TY * s);
            // the column's rows are also its exchange space: every thread has read them
            // before the first exchange writes over them
            __syncthreads();
            fft<P, N>(v, j, tw, 1, col, sg);
            // the last stage leaves the outputs in registers; every exchange read is done
#pragma unroll
            for (int s = 0; s < 8; s++) col.put(j + TY * s, v[s]);
            __syncthreads();
        }
    };

#pragma unroll 1
    for (int z = cid; z < N; z += nclusters) {   // the same planes for every CTA of the cluster
        const size_t zb = (size_t)z * N * NX + c0;
        for (int row = warp; row < N; row += NWARPS)
            for (int lc = lane; lc < ncols; lc += 32) slab[row * LDC + lc] = W[zb + (size_t)row * NX + lc];
        __syncthreads();
        if (DO_YI) y_transforms(+1);
        cluster_barrier();   // every slab holds its columns in y
        // x-lines of rows [rank RPC, (rank+1) RPC)
#pragma unroll 1
        for (int xr = 0; xr < X::XROUNDS; xr++) {
            const int li = xr * X::XLINES + tid / TX, j = tid % TX;
            const bool act = li < X::RPC;
            ClusterLine<S, N, CL> line{slab, rank * X::RPC + (act ? li : 0), act};
            LineSmem<P> lsm{xbuf + (tid / TX) * X::PADM};
            x_line_body<P, N, MODE_STEP, ClusterLine<S, N, CL>, ClusterLine<S, N, CL>>(line, line, j, lsm, tw, scale,
                                                                                      rlam, want_sum, st);
        }
        cluster_barrier();   // every remote write into this slab has landed
        y_transforms(-1);
        for (int row = warp; row < N; row += NWARPS)
            for (int lc = lane; lc < ncols; lc += 32) W[zb + (size_t)row * NX + lc] = slab[row * LDC + lc];
        __syncthreads();   // the slab is reloaded by the next plane
    }

    const unsigned long long key = block_max_key<X::NT>(st.dkey(), kred);
    if (tid == 0) part_max[blockIdx.x] = __longlong_as_double((long long)key);
    if (want_sum) {
        NSum acc;
        acc.s = st.total();
        acc.c = 0.0;
        double unused = 0.0;
        block_reduce<X::NT>(acc, unused, red);
        if (tid == 0) part_sum[blockIdx.x] = acc.value();
    }
}

}  // namespace kg
