// kg_ensemble.cuh -- one persistent launch per time step for a batch of independent
// instances of the scheme (parametric studies of blow-up, Aseeri et al. section 1),
// on grids of 64^3 and 128^3.
//
// A launch runs the four passes of a step (x, forward y, z with the update, inverse
// y) for every instance that has not blown up, separated by grid-wide barriers.
// Each pass is cut into work units of 256 threads of one instance; CTAs take units
// round-robin.  max|u^n| of each instance is gathered during the x pass; before its
// update an instance whose max exceeds the threshold is frozen at level n (no more
// updates, no more units), which is the per-instance blow-up flag.
//
// The grid barrier is a counter plus a generation word with a bounded wait: a wait
// that exceeds spin_limit polls sets status = 1 and makes every CTA leave the launch,
// so a barrier can never hang the device.
#pragma once
#include "kg_kernels.cuh"

namespace kg {

constexpr int kEnsThreads = 256;
constexpr int kEnsMaxInst = 1024;

struct EnsInst {
    double2* S0;
    double2* S1;
    void* W;
    long long level;
    long long blowup_level;
    int N;
    int phase;
    int frozen;
    int pad;
    double maxabs;       // max |u^l| seen by the last step that ran
};

struct EnsTab {
    const void* tw;
    const double2* coef;
    const double* w2;
};

struct EnsParams {
    EnsInst* inst;
    int count;
    int order;                 // 0: units in instance order; 1: largest instances first
    EnsTab tab64, tab128;
    unsigned* maxkey;          // [2][count] float-bit keys of max|u| (by step parity)
    unsigned* bar;             // [0] arrival counter, [1] generation
    int* status;               // 0 ok, 1 a barrier wait timed out
    unsigned long long* step_ctr;
    const int* order_idx;      // instance visiting order (length count)
    double lam;
    double inv_dt;
    unsigned thr_key;          // float bits of the blow-up threshold (0xffffffff: off)
    int missing;               // test hook: barriers wait for one CTA more than the grid has
    long long spin_limit;
};

// Launch schedules of the ensemble step, chosen by the autotuner (kg_ens_tune):
//   bit 0: column tiles of half the default width (64-byte instead of 128-byte rows;
//          twice the tiles per unit);
//   bit 1: the short radix stage first in transforms whose length is not a power of 8
//          (128-point columns and x-line pairs, 32-point FP32 x-lines; FftShape).
// Every schedule computes the same step; a tile width changes nothing of the arithmetic,
// the stage order changes the rounding of the transforms (double-float/FP32 level).
constexpr int kEnsSchedules = 4;
template <int SCHED>
struct EnsSched {
    static constexpr int cdiv = (SCHED & 1) ? 2 : 1;
    static constexpr bool remfirst = (SCHED & 2) != 0;
};

// work units per pass for a grid of size N (256 threads each)
template <class P, int N, int SCHED = 0>
struct EnsUnits {
    static constexpr int C = ColShape<P>::C / EnsSched<SCHED>::cdiv;
    static constexpr int TPP = (N / 2 + 1 + C - 1) / C;              // column tiles per plane
    static constexpr int TPU = kEnsThreads / (C * N / 8);             // tiles per unit
    static constexpr int col_units = (N * TPP + TPU - 1) / TPU;
    static constexpr int LPU = kEnsThreads / (N / 16);                // x-lines per unit
    static constexpr int x_units = N * N / LPU;
    static_assert(TPU >= 1 && LPU >= 1, "unit shape");
};

__device__ __forceinline__ bool ens_barrier(const EnsParams& p, unsigned nblocks) {
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        volatile unsigned* gen = p.bar + 1;
        const unsigned g = *gen;
        __threadfence();
        const unsigned expect = nblocks + (p.missing ? 1u : 0u);
        const unsigned arrived = atomicAdd(p.bar, 1u) + 1u;
        int ok = 1;
        if (arrived == expect) {
            atomicExch(p.bar, 0u);
            __threadfence();
            atomicAdd(p.bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*gen == g) {
                if (++spins > p.spin_limit || *((volatile int*)p.status) != 0) {
                    atomicExch(p.status, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        s_ok = ok && (*((volatile int*)p.status) == 0);
    }
    __syncthreads();
    return s_ok != 0;
}

template <class P, int N, int SCHED>
__device__ __forceinline__ void ens_unit(const EnsParams& p, int ii, int unit, int pass, bool active_z,
                                         int inst_phase, unsigned* maxkey_row, typename P::S* sm) {
    typedef typename P::S S;
    typedef EnsUnits<P, N, SCHED> U;
    constexpr bool RF = EnsSched<SCHED>::remfirst;
    constexpr int NH = N / 2 + 1;
    const EnsInst& in = p.inst[ii];
    const EnsTab& tb = (N == 64) ? p.tab64 : p.tab128;
    const S* tw = (const S*)tb.tw;
    S* W = (S*)in.W;
    if (pass == 0) {
        Stats<P> st;
        st.init();
        if constexpr (XPaired<P>::value) {
            // lines in pairs through one N-point transform (a pair fits in one warp here)
            typedef XpShape<N> XP;
            static_assert(!XP::CTA_SYNC, "ensemble grids keep a line pair inside a warp");
            const int pi = threadIdx.x / XP::T, jp = threadIdx.x % XP::T;
            const size_t pair = (size_t)unit * (U::LPU / 2) + pi;
            LineSmemX<P, false> lsm{sm + pi * XP::PADN, 0u, 0u};
            x_pair_body<P, N, MODE_STEP, LineSmemX<P, false>, RF>(W + 2 * pair * NH, jp, lsm, tw,
                                                                  1.0 / ((double)N * N * N), P::from_f64(p.lam),
                                                                  false, st);
        } else {
            constexpr int T = N / 16;
            const int li = threadIdx.x / T, j = threadIdx.x % T;
            const size_t line = (size_t)unit * U::LPU + li;
            LineSmem<P> lsm{sm + li * XShape<N>::PADM};
            x_line_body<P, N, MODE_STEP, const S*, S* __restrict__, RF>(W + line * NH, W + line * NH, j, lsm, tw,
                                                                        1.0 / ((double)N * N * N),
                                                                        P::from_f64(p.lam), false, st);
        }
        const unsigned k2 = st.fkey();
        const unsigned wmax = __reduce_max_sync(0xffffffffu, k2);
        if ((threadIdx.x & 31) == 0) atomicMax(maxkey_row + ii, wmax);
    } else {
        constexpr int C = U::C, T = N / 8;
        const int sub = threadIdx.x / (C * T);
        const int t = threadIdx.x % (C * T);
        const int c = t % C, j = t / C;
        const int tile = unit * U::TPU + sub;
        const bool tile_ok = tile < N * U::TPP;
        const int plane = tile_ok ? tile / U::TPP : 0;
        const int kx = (tile_ok ? tile % U::TPP : 0) * C + c;
        const bool valid = tile_ok && kx < NH;
        ColSmem<P, C> csm{sm + sub * (N * C), c};
        if (pass == 1) {
            col_body<P, P, P, N, -1, C, RF>(W, W, (size_t)plane * N * NH + kx, NH, valid, j, csm, tw);
        } else if (pass == 3) {
            col_body<P, P, P, N, +1, C, RF>(W, W, (size_t)plane * N * NH + kx, NH, valid, j, csm, tw);
        } else {
            double2* cur = inst_phase ? in.S1 : in.S0;
            double2* old = inst_phase ? in.S0 : in.S1;
            NSum q;
            q.s = 0.0;
            q.c = 0.0;
            z_body<P, N, 0, C, RF>(W, cur, old, kx, plane, valid, j, csm, tw, tb.coef, tb.w2, p.inv_dt, active_z, false,
                                   q);
        }
    }
}

// a[0] = 0 and a[1..n] hold counts on entry; on exit a[k] = sum of counts before k
// (a[n] = total).  All kEnsThreads threads call it.
__device__ __forceinline__ void block_exclusive_scan(int* a, int n) {
    __shared__ int s_warp[kEnsThreads / 32];
    constexpr int PER = (kEnsMaxInst + kEnsThreads - 1) / kEnsThreads;   // entries per thread
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int loc[PER];
    int sum = 0;
#pragma unroll
    for (int q = 0; q < PER; q++) {
        const int k = t * PER + q + 1;
        loc[q] = k <= n ? a[k] : 0;
        sum += loc[q];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
        int x = lane < kEnsThreads / 32 ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += v;
        }
        if (lane < kEnsThreads / 32) s_warp[lane] = x;
    }
    __syncthreads();
    int run = incl - sum + (w > 0 ? s_warp[w - 1] : 0);   // exclusive prefix of this thread's first entry
#pragma unroll
    for (int q = 0; q < PER; q++) {
        const int k = t * PER + q + 1;
        run += loc[q];
        if (k <= n) a[k] = run;
    }
    if (t == 0) a[0] = 0;
    __syncthreads();
}

// resident CTAs per SM the step kernel is compiled for (the autotuner picks up to this
// many): the largest count with at most a few dozen bytes of spills
template <class P>
struct EnsMinBlocks {
    static constexpr int value = 2;
};
template <>
struct EnsMinBlocks<PrecDF> {
    static constexpr int value = 3;
};
template <>
struct EnsMinBlocks<PrecF32> {
    static constexpr int value = 4;
};

template <class P, int SCHED>
__global__ void __launch_bounds__(kEnsThreads, EnsMinBlocks<P>::value) k_ens_step(EnsParams p) {
    typedef typename P::S S;
    extern __shared__ __align__(16) unsigned char smraw[];
    S* sm = reinterpret_cast<S*>(smraw);
    __shared__ int s_pref[kEnsMaxInst + 1];
    __shared__ unsigned char s_frozen0[kEnsMaxInst];
    __shared__ unsigned char s_phase0[kEnsMaxInst];
    __shared__ unsigned char s_n128[kEnsMaxInst];

    const unsigned par = (unsigned)(*((volatile unsigned long long*)p.step_ctr) & 1ull);
    unsigned* keys = p.maxkey + (size_t)par * p.count;
    for (int i = threadIdx.x; i < p.count; i += kEnsThreads) {
        s_frozen0[i] = (unsigned char)(p.inst[i].frozen != 0);
        s_phase0[i] = (unsigned char)p.inst[i].phase;
        s_n128[i] = (unsigned char)(p.inst[i].N == 128);
    }
    __syncthreads();

    for (int pass = 0; pass < 4; pass++) {
        // units of every live instance in visiting order; the z and inverse-y passes
        // skip the instances whose max|u| crossed the threshold in this step's x pass
        for (int k = threadIdx.x; k < p.count; k += kEnsThreads) {
            const int i = p.order_idx[k];
            bool live = !s_frozen0[i];
            if (pass >= 2 && live) live = !(((volatile unsigned*)keys)[i] > p.thr_key);
            int n = 0;
            if (live) {
                if (s_n128[i]) n = (pass == 0) ? EnsUnits<P, 128, SCHED>::x_units : EnsUnits<P, 128, SCHED>::col_units;
                else n = (pass == 0) ? EnsUnits<P, 64, SCHED>::x_units : EnsUnits<P, 64, SCHED>::col_units;
            }
            s_pref[k + 1] = n;
        }
        __syncthreads();
        block_exclusive_scan(s_pref, p.count);
        const int total = s_pref[p.count];
        for (int unit = blockIdx.x; unit < total; unit += gridDim.x) {
            int lo = 0, hi = p.count;   // last k with s_pref[k] <= unit
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_pref[mid] <= unit) lo = mid;
                else hi = mid;
            }
            const int ii = p.order_idx[lo];
            const int local = unit - s_pref[lo];
            if (!s_n128[ii]) ens_unit<P, 64, SCHED>(p, ii, local, pass, true, s_phase0[ii], keys, sm);
            else ens_unit<P, 128, SCHED>(p, ii, local, pass, true, s_phase0[ii], keys, sm);
            __syncthreads();
        }
        if (pass == 3) break;
        if (!ens_barrier(p, gridDim.x)) return;
        if (pass == 2 && blockIdx.x == 0) {
            // bookkeeping of the step: blow-up flags, levels, array roles, next step's keys
            unsigned* next = p.maxkey + (size_t)(par ^ 1u) * p.count;
            for (int i = threadIdx.x; i < p.count; i += kEnsThreads) {
                if (!s_frozen0[i]) {
                    const unsigned k = keys[i];
                    EnsInst& in = p.inst[i];
                    in.maxabs = (double)__uint_as_float(k);
                    if (k > p.thr_key) {
                        in.frozen = 1;
                        in.blowup_level = in.level;
                    } else {
                        in.level += 1;
                        in.phase ^= 1;
                    }
                }
                next[i] = 0u;
            }
            if (threadIdx.x == 0) *p.step_ctr += 1ull;
        }
    }
}

}  // namespace kg
